// Shared device-side definitions of the masked SpGEMM library (sm_103a).
//
// Problem (Sec. 2): C = M .* (A B) or C = !M .* (A B) over CSR operands on a
// semiring; only M's pattern is used; an output entry exists iff the mask
// allows it and at least one product was inserted (SET state, Sec. 5.1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "msgemm.h"

namespace msg {

constexpr unsigned FULL = 0xffffffffu;

// Row kinds chosen by the binning pass (one accumulator form per kind).
//   _W: one warp per row, table in a per-warp shared-memory slab
//   _B: one CTA per row, table in the CTA's shared-memory slab
//   _T: one CTA per row, dense MSA over column tiles (any n; heavy rows)
enum Kind : int {
    K_EMPTY = 0,   // no output possible (no product, or nothing allowed)
    K_MSA_W,       // Sec. 5.2 MSA, dense states + values over all n columns
    K_MSA_T,       // Sec. 5.2 MSA over column tiles (tile index of B, or cursors)
    K_HASH_W,      // Sec. 5.3 hash keyed by mask columns (load factor <= 0.5)
    K_HASH_B,
    K_MCA_W,       // Sec. 5.4 MCA: rank of j in the mask row by binary search
    K_MCA_B,
    K_DOT_W,       // Sec. 4.1 pull: per mask entry, A_i* . B_*j
    K_DOT_B,
    K_CHASH_W,     // complemented: hash keyed by produced columns
    K_CHASH_B,
    K_CMSA_T,      // complemented: MSA with NOTALLOWED default flipped, tiled
    K_CMSA_G,      // complemented, dense output: (row, tile) items over the whole grid, tile-major
    K_MSA_G,       // plain, heaviest rows of wide products: (row, tile) items, tile-major
    K_HEAP_W,      // plain: multiway merge of B rows (Sec. 5.5), NInspect = 1
    K_HEAPDOT_W,   // plain: the same with NInspect unbounded
    K_CHEAP_W,     // complemented: multiway merge, NInspect = 0
    K_MCA_Q,       // plain, tiny rows: MCA on an eight-lane team, mask row in registers
    K_DOT_Q,       // plain, tiny masks: pull on an eight-lane team, A_i* searched in global memory
    K_HASH_L,      // Sec. 5.3 hash on one CTA with a large slab: mask rows too long for K_HASH_B
    NKIND
};

// K_MCA_Q rows: at most QMASK mask entries and at most Policy.q_flops_max
// push products; K_DOT_Q rows: pull rows with at most QDMASK mask entries and
// at most Policy.q_flops_max pull pairs; QTEAM lanes per row.
constexpr int QMASK = 8, QTEAM = 8;
// K_DOT_Q: mask entries per row (QDMASK / QTEAM per lane).  32 was measured
// slower than the warp pull kernel on the batch's 16-entry mask rows: the
// team walks mask entries one after another, each a chain of dependent
// global loads, while the warp kernel searches a staged copy of A_i*.
constexpr int QDMASK = 8;

// Families (msgemm_accumulator) for preference lists.
enum Family : int { F_AUTO = 0, F_MSA = 1, F_HASH = 2, F_MCA = 3, F_DOT = 4, F_HEAP = 5, F_HEAPDOT = 6 };

// Heap kinds: one warp per row, each lane holding up to HEAP_PER_LANE row
// iterators of B in registers; rows with more stored entries of A take
// another kind.
constexpr int HEAP_PER_LANE = 4;
constexpr int HEAP_MAX_ITERS = 32 * HEAP_PER_LANE;
constexpr int HEAP_INSPECT_ALL = 0x7fffffff;   // NInspect = infinity

// One product of a (possibly batched) call.  All pointers are device pointers.
struct DevProd {
    const int *m_rp, *m_ci;                  // mask M (m x n), pattern only
    const int *a_rp, *a_ci; const void *a_v;  // A (m x k), rows enumerated
    const int *b_rp, *b_ci; const void *b_v;  // B (k x n), rows enumerated (push)
    const int *bt_rp, *bt_ci; const void *bt_v;  // B^T as CSR (n x k) for pull; may be null
    int m, n, k;
    int complement;
    int a_sorted;                             // A rows ascending (needed by DOT's search)
    long long row0;                           // first global row of this product
    long long tile0;                          // first compaction tile of this product
    long long abase;                          // first cursor slot (stored entries of A before this product)
    long long tmp0;                           // first temporary-output slot of this product (plain mask)
    const int *tpos;                          // tile index of B, tile-major planes, or null
    int tstride;                              // plane length (rows of B): row c, tile t at int2 tpos[t * tstride + c]
    int *c_rp, *c_ci; void *c_v; long long *c_nnz;  // outputs
};

// One product by value (grid-constant parameter) when by_value is set, else
// a device table (always for batches; also for a single product replayed from
// a CUDA graph, whose outputs change between replays).
struct ProdSet {
    int P;
    int by_value;
    const DevProd *tab;
    DevProd p0;
};

__device__ __forceinline__ const DevProd &prod_at(const ProdSet &ps, int p) {
    return ps.by_value ? ps.p0 : ps.tab[p];
}

// Product owning global row r (binary search over row0).
__device__ __forceinline__ int prod_of_row(const ProdSet &ps, long long r) {
    if (ps.P == 1) return 0;
    int lo = 0, hi = ps.P - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (ps.tab[mid].row0 <= r) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Product of global row r: recorded by the binning pass for batched calls
// (one load instead of a search of the product table), else searched.
__device__ __forceinline__ int row_prod(const ProdSet &ps, const int *prod, long long r) {
    return prod ? prod[r] : prod_of_row(ps, r);
}

// Per-row arrays of one pipeline run (workspace).
struct RowArrays {
    long long R;            // total rows over all products
    long long *flops;       // products per row (push: sum of |B_k*| over A_i*)
    long long *tmpoff;      // first slot of the row in the temporary output
    int *cnt;               // entries kept in the row
    unsigned char *kind;    // Kind of the row
    int *perm;              // rows grouped by kind
    int *prod;              // product of each row (batched calls; null for one product)
    int *kind_count;        // [NKIND] rows per kind
    int *kind_off;          // [NKIND + 1] exclusive offsets into perm
    int *kind_fill;         // [NKIND] scatter cursors
    int *kind_next;         // [NKIND] dynamic work cursors (heavy kinds)
    long long *bound_total; // complemented: total temporary room
    int *any_dot;           // set when a row picked the pull kernel
    int *nlong;             // binning: rows listed for the one-CTA-per-row pass
    int *gplain;            // MSA_G rows assigned so far (capped at Policy.grid_cap)
    int *sub_count;         // [NKIND * NCLS_FLOPS] rows per (kind, flops class)
    int *sub_fill;          // [NKIND * NCLS_FLOPS] scatter cursors
    unsigned *err;          // device error word
};

// Temporary output (sized by the mask for plain masks, by per-row bounds for
// complemented ones); entries of a row are stored compacted from tmpoff.
struct TmpOut {
    int *ci;
    void *v;
};

// Rows of a kind are listed heaviest first by flops class: class
// NCLS_FLOPS - 1 - min(NCLS_FLOPS - 1, floor(log2 flops)) ascending.
constexpr int NCLS_FLOPS = 32;
__device__ __forceinline__ int flops_sub(long long f) {
    const int lg = 63 - __clzll((unsigned long long)f | 1ULL);
    return NCLS_FLOPS - 1 - min(NCLS_FLOPS - 1, lg);
}

// Most MSA_G rows per call (Policy.grid_cap): their piece tables are sized on
// the host before binning, by the cap (rows beyond it take MSA_T); the cap is
// GRID_TABLE_SLOTS / tiles per row, within [GRID_CAP_MIN, GRID_CAP_MAX].
constexpr long long GRID_TABLE_SLOTS = 1LL << 24;
constexpr int GRID_CAP_MIN = 4096, GRID_CAP_MAX = 65536;
// Most column tiles of a product for the grid kinds (beyond: one CTA per row).
constexpr int GRID_MAX_TILES = 4096;

// Per-kind shared-memory budget and preference lists used by binning.
constexpr int NCLASS = 16;
struct Policy {
    int force;                    // Family, F_AUTO = per-row choice
    int allow_dot;
    float dot_ratio;              // pull when pull_cost * dot_ratio < flops
    int warp_flops_max;           // rows above go to CTA-level kinds
    int q_flops_max;              // K_MCA_Q: plain rows with <= QMASK mask entries and at most this
                                  // many push products (0: never)
    int slab[NKIND];              // bytes per warp (_W) or per CTA (_B, _T); 0 = disabled
    int tileT[2];                 // MSA_T tile width for [plain, complemented]
    int grid;                     // grid kinds: 0 off, 1 by the rules below, 2 for every heavy row
    int comp_grid_all;            // grid 1: every heavy complemented row (the full rooms fit), not only dense ones
    long long grid_min_flops;     // MSA_G: CTA rows with at least this much push work (grid 1)
    int grid_cap;                 // MSA_G: most rows per call
    unsigned char pref[NCLASS][4];  // families in preference order (F_AUTO = end)
};

__host__ __device__ __forceinline__ int row_class(long long flops, int mnz) {
    int fb = flops <= 512 ? 0 : flops <= 8192 ? 1 : flops <= 131072 ? 2 : 3;
    int mb = mnz <= 8 ? 0 : mnz <= 64 ? 1 : mnz <= 512 ? 2 : 3;
    return fb * 4 + mb;
}

// Device error bits.
enum : unsigned {
    ERR_TIMEOUT = 1u,
    ERR_INVALID = 2u,
    ERR_UNSORTED = 4u,
    ERR_INTERNAL = 8u,
};

// ------------------------------------------------------------------ semirings
// acc_t: shared-memory accumulator; out_t: stored result; in_t: input value.
template <int SR> struct Sr;

template <> struct Sr<MSGEMM_PLUS_TIMES_F32> {
    using in_t = float;
    using acc_t = float;
    using out_t = float;
    static constexpr bool vals = true;      // inputs carry values
    static constexpr bool count_set = false;  // SET state kept in a bit array
    __device__ static __forceinline__ acc_t mul(in_t a, in_t b) { return a * b; }
    __device__ static __forceinline__ void add(acc_t *p, acc_t v) { atomicAdd(p, v); }
    __device__ static __forceinline__ out_t out(acc_t v) { return v; }
};

template <> struct Sr<MSGEMM_PLUS_TIMES_I64> {
    using in_t = long long;
    using acc_t = unsigned long long;
    using out_t = long long;
    static constexpr bool vals = true;
    static constexpr bool count_set = false;
    __device__ static __forceinline__ acc_t mul(in_t a, in_t b) {
        return (unsigned long long)a * (unsigned long long)b;  // wraps mod 2^64
    }
    // Shared-memory add mod 2^64 as two 32-bit atomics (64-bit shared atomics
    // are about 9x slower): the low word is added and its old value returned;
    // if that add wrapped, one carry goes to the high word with the addend's
    // high half.  Every wrap is counted by exactly the add that caused it, so
    // the final 64-bit value is the exact sum mod 2^64 in any order.
    __device__ static __forceinline__ void add(acc_t *p, acc_t v) {
        unsigned *w = reinterpret_cast<unsigned *>(p);   // little-endian: w[0] low, w[1] high
        const unsigned lo = (unsigned)v;
        const unsigned old = atomicAdd(w, lo);
        const unsigned hi = (unsigned)(v >> 32) + (old + lo < old ? 1u : 0u);
        if (hi) atomicAdd(w + 1, hi);
    }
    __device__ static __forceinline__ out_t out(acc_t v) { return (long long)v; }
};

// plus-pair: a count per entry, at most |A_i*| < 2^31, so 32 bits never wrap.
template <> struct Sr<MSGEMM_PLUS_PAIR_I64> {
    struct none_t {};
    using in_t = none_t;
    using acc_t = unsigned int;
    using out_t = long long;
    static constexpr bool vals = false;
    static constexpr bool count_set = true;   // count > 0 <=> SET
    __device__ static __forceinline__ acc_t mul(in_t, in_t) { return 1u; }
    __device__ static __forceinline__ void add(acc_t *p, acc_t v) { atomicAdd(p, v); }
    __device__ static __forceinline__ out_t out(acc_t v) { return (long long)v; }
};

template <int SR>
__device__ __forceinline__ typename Sr<SR>::in_t load_val(const void *base, long long idx) {
    if constexpr (Sr<SR>::vals) {
        // a pattern operand (no value array) has every stored value 1
        using in_t = typename Sr<SR>::in_t;
        return base ? __ldg(static_cast<const in_t *>(base) + idx) : in_t(1);
    } else {
        return typename Sr<SR>::in_t{};
    }
}

// Accumulator of the column-tiled MSA kinds.  int64 keeps only the low
// 32-bit word per column in shared memory (so its tiles are as wide as the
// 32-bit semirings'); the high word lives in a per-CTA global array `hi` of
// one word per tile column, touched only by products whose high half is
// non-zero and by low-word carries.  As for the two-word shared add, every
// wrap of the low word is counted once by the add that caused it, so
// lo + 2^32 hi is the exact sum mod 2^64 in any order.  `get` reads a column,
// `clear` zeroes it (both words), `take` does both.  hi is read through L2:
// its words are changed by global atomics.
template <int SR> struct TileAcc {
    using acc_t = typename Sr<SR>::acc_t;
    using lo_t = acc_t;
    static constexpr bool split = false;
    __device__ static __forceinline__ void add(lo_t *lo, unsigned *, int jj, acc_t v) { Sr<SR>::add(&lo[jj], v); }
    __device__ static __forceinline__ acc_t get(const lo_t *lo, const unsigned *, int jj) { return lo[jj]; }
    __device__ static __forceinline__ void clear(lo_t *lo, unsigned *, int jj) { lo[jj] = 0; }
    __device__ static __forceinline__ acc_t take(lo_t *lo, unsigned *, int jj) {
        const acc_t v = lo[jj];
        lo[jj] = 0;
        return v;
    }
};
template <> struct TileAcc<MSGEMM_PLUS_TIMES_I64> {
    using acc_t = unsigned long long;
    using lo_t = unsigned;
    static constexpr bool split = true;
    __device__ static __forceinline__ void add(lo_t *lo, unsigned *hi, int jj, acc_t v) {
        const unsigned l = (unsigned)v;
        const unsigned old = atomicAdd(&lo[jj], l);
        const unsigned h = (unsigned)(v >> 32) + (old + l < old ? 1u : 0u);
        if (h) atomicAdd(&hi[jj], h);
    }
    __device__ static __forceinline__ acc_t get(const lo_t *lo, const unsigned *hi, int jj) {
        return ((acc_t)__ldcg(hi + jj) << 32) | lo[jj];
    }
    __device__ static __forceinline__ void clear(lo_t *lo, unsigned *hi, int jj) {
        lo[jj] = 0;
        if (__ldcg(hi + jj)) hi[jj] = 0;
    }
    __device__ static __forceinline__ acc_t take(lo_t *lo, unsigned *hi, int jj) {
        const unsigned h = __ldcg(hi + jj);
        const acc_t v = ((acc_t)h << 32) | lo[jj];
        lo[jj] = 0;
        if (h) hi[jj] = 0;
        return v;
    }
};
// Shared bytes per column of a tiled accumulator's value array: 4 for every
// semiring (fp32, 32-bit plus-pair counts, the low word of int64).
constexpr int TILE_ACC_BYTES = 4;

template <int SR> struct SrSizes {
    static constexpr int acc = sizeof(typename Sr<SR>::acc_t);
    static constexpr int in = Sr<SR>::vals ? (int)sizeof(typename Sr<SR>::in_t) : 0;
    static constexpr int out = sizeof(typename Sr<SR>::out_t);
    static constexpr bool setbits = !Sr<SR>::count_set;
};

// ------------------------------------------------------------------ sizing
__host__ __device__ __forceinline__ long long pow2_at_least(long long x) {
    long long p = 32;
    while (p < x) p <<= 1;
    return p;
}
__host__ __device__ __forceinline__ long long align8(long long x) { return (x + 7) & ~7LL; }
__host__ __device__ __forceinline__ long long words32(long long bits) { return (bits + 31) >> 5; }

// Hash (mask-keyed) table: per slot a 32-bit key (the mask column; bit 31
// marks the SET state where the semiring keeps one) and the slot's
// accumulator.  Slots: the power of two at or above 4 x nnz(m) (load factor
// at most 0.25, Sec. 5.3), at least 32, halved while the slab is too small
// and the load stays at most 0.5.  Returns 0 if the row does not fit.
__host__ __device__ __forceinline__ long long hash_table_bytes(long long H, int acc) {
    return align8(4 * H) + H * acc;   // keys, then the (8-byte aligned) accumulators
}
__host__ __device__ __forceinline__ long long hash_slots(long long mnz, int acc, long long slab) {
    // a power of two: 4 nnz(m) slots (load 1/4), halved toward load 1/2 to fit the slab
    if (mnz <= 0 || mnz > (1 << 24)) return 0;
    long long h = 32;
    while (h < 4 * mnz) h <<= 1;
    while (h / 2 >= 2 * mnz && hash_table_bytes(h, acc) > slab) h >>= 1;
    return hash_table_bytes(h, acc) <= slab ? h : 0;
}

// Two-choice (cuckoo) positions of key x in a table of H = 2^lg >= 32 slots,
// from one multiply u = x * c (mod 2^32): p1 = the top lg bits of u, and
// p2 = p1 xor (d | 1) with d the next lg bits of u, so p2 != p1 and either
// position gives the other from the key alone (the partial-key form of
// Fan et al.'s cuckoo filters).  Every key of a built table sits at one of its
// two positions, so a lookup reads exactly two slots (Pagh and Rodler's
// cuckoo hashing; parallel insertion by atomic exchange as in Alcantara et
// al.'s GPU hash tables).
struct CuckooHash {
    unsigned c, H, s1, s2;   // s1 = 32 - lg, s2 = 32 - 2 lg (0 when 2 lg > 32)
    __device__ __forceinline__ void pos(unsigned x, unsigned &p1, unsigned &p2) const {
        const unsigned u = x * c;
        p1 = u >> s1;
        p2 = p1 ^ (((u >> s2) & (H - 1u)) | 1u);
    }
    __device__ __forceinline__ unsigned h1(unsigned x) const { return (x * c) >> s1; }
};
__host__ __device__ __forceinline__ CuckooHash cuckoo_hash(unsigned c, unsigned H) {
    unsigned lg = 0;
    while ((1u << lg) < H) ++lg;
    return CuckooHash{c, H, 32u - lg, 2 * lg < 32 ? 32u - 2 * lg : 0u};
}
// Multipliers of the first attempt and of the retry (odd constants).
constexpr unsigned CUCKOO_A = 0x9E3779B1u, CUCKOO_B = 0xC2B2AE3Du;
constexpr int CUCKOO_KICKS = 64;
__host__ __device__ __forceinline__ long long mca_bytes(long long mnz, int acc, bool setbits) {
    return align8(4 * mnz) + align8(mnz * acc) + (setbits ? 4 * words32(mnz) : 0);
}
__host__ __device__ __forceinline__ long long dot_bytes(long long anz, long long mnz, int in, int acc, bool setbits) {
    return align8(4 * anz) + align8(anz * in) + align8(mnz * acc) + (setbits ? 4 * words32(mnz) : 0);
}
__host__ __device__ __forceinline__ long long msa_bytes(long long ncols, int acc) {
    return align8(ncols * acc) + 8 * words32(ncols);
}
// Complemented hash: keys + values for >= 2 x bound slots, plus the sorted
// mask row for membership tests.  Returns slots or 0.
__host__ __device__ __forceinline__ long long chash_slots(long long bound, long long mnz, int acc, long long slab) {
    long long h = pow2_at_least(2 * bound);
    long long bytes = align8(4 * h) + align8(h * acc) + align8(4 * mnz);
    return bytes <= slab ? h : 0;
}
// MSA_T tile width for a slab: values + two bit arrays, multiple of 32.
__host__ __device__ __forceinline__ int msa_tile_width(long long slab, int acc) {
    long long t = (slab - 64) * 32 / (32 * acc + 8);
    t &= ~31LL;
    return t > 0 ? (int)t : 0;
}

// ------------------------------------------------------------------ barriers
// Block barrier after divergent work: lanes leave data-dependent loops (a
// probe chain inside a product callback, a per-lane range walk) at different
// times, so each warp first reconverges (__syncwarp) and then meets the
// other warps.
__device__ __forceinline__ void block_sync() {
    __syncwarp();
    __syncthreads();
}

// Read of a shared-memory word that other threads of the team set with
// atomics before the last team barrier, as a volatile load: the compiler
// neither reuses an earlier read of the word nor moves the read.  With plain
// loads, the linear-probe lookups of CTA hash rows missed keys that the build
// had inserted before the barrier: now and then at first, and in every run
// once the team barrier reconverged the warp first; with volatile loads none
// did.
template <class T> __device__ __forceinline__ T ld_vol(const T *p) {
    return *static_cast<const volatile T *>(p);
}

// ------------------------------------------------------------------ teams
// A team cooperates on one row: one warp (_W kinds) or the whole CTA.
template <bool CTA> struct Team {
    __device__ __forceinline__ int tid() const { return CTA ? (int)threadIdx.x : (int)(threadIdx.x & 31); }
    __device__ __forceinline__ int size() const { return CTA ? (int)blockDim.x : 32; }
    __device__ __forceinline__ int warp() const { return CTA ? (int)(threadIdx.x >> 5) : 0; }
    __device__ __forceinline__ int nwarps() const { return CTA ? (int)(blockDim.x >> 5) : 1; }
    // Barrier that also publishes the team's shared-memory atomics (hash
    // keys, bitmaps, accumulators) to the plain loads that follow it: the
    // warp reconverges, fences its shared-memory writes, then meets the
    // other warps (block_sync).
    __device__ __forceinline__ void sync() const {
        if (CTA) {
            __syncwarp();
            __threadfence_block();
            __syncthreads();
        } else {
            __threadfence_block();
            __syncwarp();
        }
    }
};

// Staging of a CSR row segment (n elements of E = 4 or 8 bytes) from global
// into shared memory by asynchronous copies (cp.async, one element per thread
// and step, so any start of the row is fine): the loads stay in flight while
// the team clears its accumulators.  Each thread then waits for its own
// copies with stage_wait(); the team barrier that follows publishes them.
template <int E, bool CTA>
__device__ __forceinline__ void stage_async(void *dst, const void *src, int n) {
    Team<CTA> team;
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *s = static_cast<const char *>(src);
    for (int q = team.tid(); q < n; q += team.size()) {
        if constexpr (E == 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + 4u * q), "l"(s + 4LL * q) : "memory");
        else
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + 8u * q), "l"(s + 8LL * q) : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void stage_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void cta_sync() {
    __syncwarp();
    __threadfence_block();
    __syncthreads();
}

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ unsigned lanemask_lt() { return (1u << lane_id()) - 1u; }

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Exclusive scan of one int per thread over the CTA; `scratch` holds >= 33 ints.
// Returns the exclusive prefix; *total receives the CTA sum.
__device__ __forceinline__ int block_excl_scan(int v, int *scratch, int *total) {
    const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int incl = warp_incl_scan(v);
    if (lane == 31) scratch[w] = incl;
    block_sync();
    if (w == 0) {
        int x = lane < nw ? scratch[lane] : 0;
        int xi = warp_incl_scan(x);
        if (lane < nw) scratch[lane] = xi - x;
        if (lane == 31) scratch[32] = xi;
    }
    block_sync();
    int res = scratch[w] + incl - v;
    *total = scratch[32];
    block_sync();
    return res;
}

__device__ __forceinline__ unsigned hash32(unsigned key, int logH) {
    return (key * 0x9E3779B1u) >> (32 - logH);
}

__host__ __device__ __forceinline__ int ilog2(long long x) {
    int l = 0;
    while ((1LL << l) < x) ++l;
    return l;
}

}  // namespace msg
