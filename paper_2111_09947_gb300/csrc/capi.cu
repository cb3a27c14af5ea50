// C ABI of the masked SpGEMM library (declarations and contracts in
// include/msgemm.h): the handle, its workspace, and the host side of the
// one-phase pipeline  validate -> bin -> [transpose for pull] -> accumulate
// per kind -> count -> compact  (Sec. 4-6).
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "launch.h"
#include "rows.cuh"

using namespace msg;

namespace {

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct msgemm_handle {
    int device = 0;
    int nsm = 0;
    int smem_optin = 0;
    cudaStream_t stream = nullptr;
    msgemm_alloc_fn alloc = nullptr;
    msgemm_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    // workspace, reused across calls
    Buf rows, small, tmp, bt, cur, prods, tix, gbuf, thi, gpbuf;
    unsigned *d_err = nullptr;   // in `small`, persistent
    int force = 0, validate = 0, allow_dot = 1, tile_index = 1, grid = 1;
    int phases = 1;   // 1: one-phase, 2: symbolic + numeric (MSGEMM_OPT_PHASES)
    int hash_kicks = CUCKOO_KICKS;   // MSGEMM_OPT_HASH_KICKS
    long long tile_index_budget = 4LL << 30;   // bytes
    // complemented rows on the grid take a room of all their open columns;
    // when those rooms of every complemented row fit this, sparse rows take
    // the grid too instead of one CTA walking all their tiles
    long long comp_room_budget = 16LL << 30;   // bytes
    unsigned char pref[NCLASS][4];
    float dot_ratio = 2.0f;
    int warp_flops_max = 65536;
    int q_flops_max = 1024;   // MSGEMM_OPT_QTEAM_FLOPS: K_MCA_Q rows (0: never)
    int warp_slab = 4608;   // shared bytes per warp of the one-warp MCA and pull kinds
    int hash_slab = 4608;   // shared bytes per warp of the one-warp hash kinds
    long long grid_min_flops = 1LL << 20;   // MSA_G: plain CTA rows with at least this push work
    int *last_kind_count = nullptr;
    unsigned char *last_kind = nullptr;
    long long last_R = 0;
    std::string last_error;
    // phase profiling (MSGEMM_OPT_PROFILE)
    int profile = 0;
    struct Phase { std::string name; cudaEvent_t a = nullptr, b = nullptr; };
    std::vector<Phase> prof;
    int nprof = 0;
    // host staging
    std::vector<DevProd> hprods;
    // CUDA graph of the last graph-mode plan (msgemm_run_batched, use_graph)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::string gkey;
    long long gkernels = 0, gcaptures = 0;
    // output allocations of the current call (the autotuner frees them)
    std::vector<void *> out_allocs;
};

namespace {

msgemm_status fail(msgemm_handle *h, msgemm_status st, const char *fmt, ...) {
    if (h) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        h->last_error = buf;
    }
    return st;
}

#define CK(call)                                                                                 \
    do {                                                                                         \
        cudaError_t e_ = (call);                                                                 \
        if (e_ != cudaSuccess)                                                                   \
            return fail(h, MSGEMM_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                     \
    } while (0)

#define CKS(expr)                            \
    do {                                     \
        msgemm_status s_ = (expr);           \
        if (s_ != MSGEMM_OK) return s_;      \
    } while (0)

void *dev_alloc(msgemm_handle *h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    if (h->alloc) return h->alloc(bytes, h->ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(msgemm_handle *h, void *p) {
    if (!p) return;
    if (h->free_fn) h->free_fn(p, h->ctx);
    else cudaFree(p);
}

// Output arrays of several products from ONE allocation: slices of the given
// byte sizes (each at least one byte, 16-byte aligned) of a single callback
// allocation, whose base is the first slice.  All null if it failed.
std::vector<char *> carve_alloc(msgemm_handle *h, const std::vector<size_t> &sizes) {
    std::vector<char *> out(sizes.size(), nullptr);
    if (sizes.empty()) return out;
    std::vector<size_t> off(sizes.size());
    size_t total = 0;
    for (size_t i = 0; i < sizes.size(); ++i) {
        off[i] = total;
        total += (std::max<size_t>(sizes[i], 1) + 15) & ~size_t(15);
    }
    char *base = static_cast<char *>(dev_alloc(h, total));
    if (!base) return out;
    h->out_allocs.push_back(base);
    for (size_t i = 0; i < sizes.size(); ++i) out[i] = base + off[i];
    return out;
}

msgemm_status grow(msgemm_handle *h, Buf &b, size_t bytes) {
    if (b.cap >= bytes && b.p) return MSGEMM_OK;
    size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    dev_free(h, b.p);
    b.p = dev_alloc(h, want);
    b.cap = b.p ? want : 0;
    if (!b.p) return fail(h, MSGEMM_ERR_OOM, "workspace allocation of %zu bytes failed", want);
    return MSGEMM_OK;
}

// Records events around a phase on the handle's stream when profiling is on.
struct PScope {
    msgemm_handle *h;
    int idx = -1;
    PScope(msgemm_handle *h_, const char *name) : h(h_) {
        if (!h->profile) return;
        if (h->nprof == (int)h->prof.size()) {
            h->prof.emplace_back();
            cudaEventCreate(&h->prof.back().a);
            cudaEventCreate(&h->prof.back().b);
        }
        idx = h->nprof++;
        h->prof[idx].name = name;
        cudaEventRecord(h->prof[idx].a, h->stream);
    }
    ~PScope() {
        if (idx >= 0) cudaEventRecord(h->prof[idx].b, h->stream);
    }
};

const char *kind_name(int k) {
    static const char *names[NKIND] = {"empty", "msa_w", "msa_t", "hash_w", "hash_b", "mca_w",
                                       "mca_b", "dot_w", "dot_b", "chash_w", "chash_b", "cmsa_t", "cmsa_g", "msa_g",
                                       "heap_w", "heapdot_w", "cheap_w", "mca_q", "dot_q", "hash_l"};
    return (k >= 0 && k < NKIND) ? names[k] : "?";
}

// Bump carving of a buffer.
struct Carver {
    char *base;
    size_t off = 0;
    explicit Carver(void *p) : base(static_cast<char *>(p)) {}
    template <class T> T *take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T *r = reinterpret_cast<T *>(base + off);
        off += count * sizeof(T);
        return r;
    }
};
template <class T> size_t carve_size(size_t count) { return ((count * sizeof(T)) + 255) & ~size_t(255); }

int acc_bytes(msgemm_semiring sr) { return sr == MSGEMM_PLUS_TIMES_I64 ? 8 : 4; }
int in_bytes(msgemm_semiring sr) { return sr == MSGEMM_PLUS_TIMES_F32 ? 4 : sr == MSGEMM_PLUS_TIMES_I64 ? 8 : 0; }
int out_bytes(msgemm_semiring sr) { return sr == MSGEMM_PLUS_TIMES_F32 ? 4 : 8; }

// Default family order per row class (flops band fb = c / 4, mask band
// mb = c % 4).  MCA first for small masks, and for rows with few products
// (fb <= 1: at most 8192) and masks up to 512 entries, whose cost is mostly
// the accumulator's setup -- copying the mask row is cheaper than building a
// hash table (an Erdos-Renyi sweep of n 2^12..2^20 and degrees 4..64 x 1..256
// had MCA ahead of hash on nearly every such point, by up to 4x); hash first
// for heavier rows.
// Default class preferences (row_class: flop bands <= 512, <= 8192, <= 131072,
// above; mask bands <= 8, <= 64, <= 512, above): MSA where the dense row
// fits a warp, then MCA for mask rows of at most 8 entries and for rows of at
// most 512 push products with mask rows up to 512 entries (setup dominates:
// MCA clears nnz(m) values, the hash table 4 nnz(m) slots), hash otherwise
// (two shared loads per product against MCA's log2 nnz(m) search steps).
// From the Erdos-Renyi density sweep (bench.py --sweep er).
void default_pref(unsigned char pref[NCLASS][4]) {
    for (int c = 0; c < NCLASS; ++c) {
        const int fb = c / 4, mb = c % 4;
        if (mb == 0 || (fb == 0 && mb <= 2)) { pref[c][0] = F_MSA; pref[c][1] = F_MCA; pref[c][2] = F_HASH; }
        else { pref[c][0] = F_MSA; pref[c][1] = F_HASH; pref[c][2] = F_MCA; }
        pref[c][3] = F_AUTO;
    }
}

Policy make_policy(const msgemm_handle *h, msgemm_semiring sr, int max_n) {
    Policy p{};
    p.force = h->force;
    p.allow_dot = h->allow_dot;
    p.dot_ratio = h->dot_ratio;
    p.warp_flops_max = h->warp_flops_max;
    p.q_flops_max = h->q_flops_max;
    const int acc = acc_bytes(sr);
    const int wslab = h->warp_slab;   // default 4.5 KB: 8 warps x 4.5 KB = 36 KB per CTA, 6 CTAs per SM
    const int hslab = h->hash_slab;
    const int bslab = 32 * 1024;  // per CTA-row: 7 CTAs per SM
    const int lslab = 96 * 1024;  // hash rows too long for bslab: 2 CTAs per SM
    const int tslab = std::min(h->smem_optin - 4096, 216 * 1024) & ~1023;
    p.slab[K_MCA_W] = p.slab[K_DOT_W] = wslab;
    p.slab[K_HASH_W] = p.slab[K_CHASH_W] = hslab;
    p.slab[K_HASH_B] = p.slab[K_MCA_B] = p.slab[K_DOT_B] = p.slab[K_CHASH_B] = bslab;
    p.slab[K_HASH_L] = lslab;
    const long long msaw = (msa_bytes(max_n, acc) + 15) & ~15LL;
    p.slab[K_MSA_W] = msaw <= 24 * 1024 ? (int)msaw : 0;
    p.slab[K_MSA_T] = p.slab[K_CMSA_T] = p.slab[K_CMSA_G] = p.slab[K_MSA_G] = tslab;
    p.grid = h->grid;
    p.grid_min_flops = h->grid_min_flops;
    p.tileT[0] = p.tileT[1] = msa_tile_width(tslab, TILE_ACC_BYTES);
    memcpy(p.pref, h->pref, sizeof p.pref);
    return p;
}

msgemm_status check_csr(msgemm_handle *h, const msgemm_csr *X, const char *name, bool need_vals) {
    if (!X) return fail(h, MSGEMM_ERR_INVALID, "%s is NULL", name);
    if (X->nrows < 0 || X->ncols < 0 || X->nnz < 0) return fail(h, MSGEMM_ERR_INVALID, "%s has a negative size", name);
    if (X->nnz >= (1LL << 31)) return fail(h, MSGEMM_ERR_OVERFLOW, "%s has nnz >= 2^31", name);
    if (!X->rowptr) return fail(h, MSGEMM_ERR_INVALID, "%s.rowptr is NULL", name);
    if (X->nnz > 0 && !X->colidx) return fail(h, MSGEMM_ERR_INVALID, "%s.colidx is NULL", name);
    if (need_vals && X->nnz > 0 && !X->values) return fail(h, MSGEMM_ERR_INVALID, "%s.values is NULL", name);
    return MSGEMM_OK;
}

// One product of a pipeline run, host view.
struct ProdIn {
    const msgemm_csr *M, *A, *B;
    int comp;
    const int *bt_rp = nullptr, *bt_ci = nullptr;  // prebuilt B^T (pull), optional
    const void *bt_v = nullptr;
    int a_sorted = 1;
    msgemm_csr_out *C = nullptr;   // compacted output
    void *aligned_out = nullptr;   // gradient form: values at the mask's slots
};

// Device check of user inputs (row pointers, column range, strict order);
// synchronises.  Internal operands (transposes with unsorted rows) never pass here.
msgemm_status validate_inputs(msgemm_handle *h, const std::vector<const msgemm_csr *> &mats) {
    cudaStream_t st = h->stream;
    for (const msgemm_csr *X : mats)
        if (X->nrows > 0) CK(launch_validate(X->rowptr, X->colidx, X->nrows, X->ncols, X->nnz, h->d_err, st, h->nsm));
    unsigned herr = 0;
    CK(cudaMemcpyAsync(&herr, h->d_err, sizeof herr, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (herr) {
        CK(cudaMemsetAsync(h->d_err, 0, sizeof herr, st));
        if (herr & ERR_UNSORTED) return fail(h, MSGEMM_ERR_UNSORTED, "an input row is not strictly ascending");
        return fail(h, MSGEMM_ERR_INVALID, "invalid row pointers or column indices");
    }
    return MSGEMM_OK;
}

// Host view of one pipeline run: workspace carved, tables built and every
// pointer the device sequence needs fixed before its first kernel.  With
// plain masks nothing in the device sequence depends on device results, so
// it can be captured once into a CUDA graph and replayed.
struct Plan {
    int P = 0;
    bool aligned = false, any_comp = false;
    msgemm_semiring sr{};
    Policy pol{};
    ProdSet ps{};
    long long R = 0, nnzA = 0, tmpn = 0, ntiles = 0, cap = 0;
    long long *room = nullptr, *tile_sums = nullptr, *tile_offs = nullptr, *chunk_start = nullptr,
              *prod_tot = nullptr, *room_tiles = nullptr;
    DevProd *dtab = nullptr;
    char *zero_begin = nullptr;
    size_t zero_bytes = 0;
    // B^T of the products whose rows may take the pull kernel
    std::vector<BtDesc> bd;
    long long bt_counts = 0, bt_nnz = 0, bt_rows = 0;
    int *bt_rp_all = nullptr, *bt_cur = nullptr, *bt_ci = nullptr;
    void *bt_v = nullptr;
    BtDesc *bt_tab = nullptr;
    long long *bt_tb = nullptr;
    // tile index of B for column-tiled products (nts[p] tiles, 0 = untiled)
    std::vector<int> nts;
    std::vector<int *> tpos;
    int gnt = 0;   // grid kinds: most column tiles of a product
    size_t gp_done_bytes = 0;   // MSA_G: per-row completion counts to zero
    size_t thi_bytes = 0;   // int64 tiled kinds: high-word arrays to zero
    RowLaunch L{};
    std::vector<int> kinds;
};

msgemm_status plan_prepare(msgemm_handle *h, std::vector<ProdIn> &in, msgemm_semiring sr, bool build_bt,
                           bool by_value, Plan &pl, bool two_phase = false) {
    const int P = (int)in.size();
    pl.P = P;
    pl.sr = sr;
    pl.aligned = P > 0 && in[0].aligned_out != nullptr;
    int max_n = 0;
    bool any_tiled = false;
    const Policy pol0 = make_policy(h, sr, 0);
    std::vector<DevProd> &dp = h->hprods;
    dp.assign(P, DevProd{});
    for (int p = 0; p < P; ++p) {
        const ProdIn &x = in[p];
        DevProd &d = dp[p];
        d.m_rp = x.M->rowptr; d.m_ci = x.M->colidx;
        d.a_rp = x.A->rowptr; d.a_ci = x.A->colidx; d.a_v = x.A->values;
        d.b_rp = x.B->rowptr; d.b_ci = x.B->colidx; d.b_v = x.B->values;
        d.bt_rp = x.bt_rp; d.bt_ci = x.bt_ci; d.bt_v = x.bt_v;
        d.m = x.M->nrows; d.n = x.M->ncols; d.k = x.A->ncols;
        d.complement = x.comp;
        d.a_sorted = x.a_sorted;
        d.row0 = pl.R;
        d.tile0 = pl.ntiles;
        d.abase = pl.nnzA;
        d.tmp0 = pl.tmpn;
        pl.R += d.m;
        pl.nnzA += x.A->nnz;
        pl.ntiles += (d.m + CTILE - 1) / CTILE;
        if (!x.comp) pl.tmpn += x.M->nnz;
        pl.any_comp |= x.comp != 0;
        max_n = std::max(max_n, d.n);
        if (d.n > pol0.tileT[x.comp ? 1 : 0]) any_tiled = true;
        pl.gnt = std::max(pl.gnt, std::min(GRID_MAX_TILES, (d.n + pol0.tileT[0] - 1) / pol0.tileT[0]));
        if (x.C) {
            d.c_rp = x.C->rowptr; d.c_ci = x.C->colidx; d.c_v = x.C->values; d.c_nnz = reinterpret_cast<long long *>(x.C->d_nnz);
            if (!x.comp) pl.cap += x.C->capacity;
        }
    }
    const long long R = pl.R, ntiles = pl.ntiles;
    if (R >= (1LL << 31)) return fail(h, MSGEMM_ERR_OVERFLOW, "total rows >= 2^31");
    pl.pol = make_policy(h, sr, max_n);
    if (two_phase) pl.pol.grid = 0;   // grid pieces need a temporary's room
    {
        double comp_room = 0.0;   // bytes if every complemented row took its full room
        for (int p = 0; p < P; ++p)
            if (in[p].comp) comp_room += (double)in[p].M->nrows * in[p].M->ncols * (4 + out_bytes(sr));
        pl.pol.comp_grid_all = comp_room <= (double)h->comp_room_budget;
    }

    // ---- per-row workspace
    const size_t rows_bytes = carve_size<long long>(R) * 3 + carve_size<int>(R) * 3 + carve_size<unsigned char>(R) +
                              carve_size<long long>(ntiles) * 3 + 256 + carve_size<long long>(2 * (size_t)P) +
                              carve_size<long long>((R + STILE - 1) / STILE + 2) + carve_size<DevProd>(P) + 4096;
    CKS(grow(h, h->rows, rows_bytes));
    Carver cv(h->rows.p);
    RowArrays &ra = pl.L.ra;
    ra.R = R;
    ra.flops = cv.take<long long>(R);
    ra.tmpoff = cv.take<long long>(R);
    pl.room = cv.take<long long>(R);
    ra.cnt = cv.take<int>(R);
    ra.perm = cv.take<int>(R);
    ra.prod = P > 1 ? cv.take<int>(R) : nullptr;
    ra.kind = cv.take<unsigned char>(R);
    pl.tile_sums = cv.take<long long>(ntiles);
    pl.tile_offs = cv.take<long long>(ntiles);
    pl.chunk_start = cv.take<long long>(ntiles + 1);
    pl.prod_tot = cv.take<long long>(2 * (size_t)P);
    pl.room_tiles = cv.take<long long>((R + STILE - 1) / STILE + 2);
    pl.dtab = cv.take<DevProd>(P);
    // small counters: zeroed per run (err is persistent, kept first)
    Carver cs(h->small.p);
    ra.err = cs.take<unsigned>(1);
    pl.zero_begin = cs.base + ((cs.off + 255) & ~size_t(255));
    ra.kind_count = cs.take<int>(NKIND);
    ra.kind_fill = cs.take<int>(NKIND);
    ra.kind_next = cs.take<int>(NKIND);
    ra.kind_off = cs.take<int>(NKIND + 1);
    ra.any_dot = cs.take<int>(1);
    ra.nlong = cs.take<int>(1);
    ra.sub_count = cs.take<int>(NKIND * NCLS_FLOPS);
    ra.sub_fill = cs.take<int>(NKIND * NCLS_FLOPS);
    ra.bound_total = cs.take<long long>(1);
    pl.L.g[0].next = cs.take<unsigned long long>(1);
    pl.L.g[1].next = cs.take<unsigned long long>(1);
    ra.gplain = cs.take<int>(1);
    pl.L.spec_off = cs.take<int>(1);
    pl.L.gnt = pl.gnt;
    pl.zero_bytes = (size_t)(cs.base + cs.off - pl.zero_begin);
    h->last_kind_count = ra.kind_count;
    h->last_kind = ra.kind;
    h->last_R = R;

    // ---- B^T for the pull kernel: row pointers in the front of the sequence,
    // entries only if some row picked it.  Building B^T costs a pass over B;
    // for one product it pays only where the pull work (mask entries x
    // average column length of B) is below half the push work (entries of A
    // x average row length of B) and the push work is at least 32x B's
    // entries (thresholds from an Erdos-Renyi sweep), or when DOT is forced.  Batches always get
    // the row pointers (one pass over all their B's together): averages miss
    // the skew of graphs whose hubs are shared by A's columns and B's rows,
    // where push work per row far exceeds the estimate, and the binning's
    // exact per-row costs then decide.
    auto want_bt = [&](const ProdIn &x) {
        if (x.comp || x.bt_rp || !x.a_sorted) return false;
        if (h->force == F_DOT || P > 1) return true;
        const double bnz = (double)x.B->nnz;
        const double push = (double)x.A->nnz * bnz / std::max(1, x.B->nrows);
        const double pull = (double)x.M->nnz * bnz / std::max(1, x.B->ncols);
        // B^T costs passes over B: only products with far more push work
        // than B's entries amortise it
        return pull * 2.0 < push && push >= 32.0 * bnz;
    };
    if (build_bt && h->allow_dot && (h->force == F_AUTO || h->force == F_DOT)) {
        for (int p = 0; p < P; ++p) {
            if (!want_bt(in[p])) continue;
            const msgemm_csr *B = in[p].B;
            pl.bd.push_back(BtDesc{B->rowptr, B->colidx, B->values, B->nrows, B->ncols, B->nnz, pl.bt_counts,
                                   pl.bt_nnz, pl.bt_rows});
            pl.bt_counts += (long long)B->ncols + 1;
            pl.bt_nnz += B->nnz;
            pl.bt_rows += B->nrows;
        }
    }
    if (!pl.bd.empty()) {
        const int Q = (int)pl.bd.size();
        const size_t bytes = carve_size<int>(pl.bt_counts + 1) * 2 + carve_size<int>(pl.bt_nnz) +
                             carve_size<char>((size_t)pl.bt_nnz * in_bytes(sr)) +
                             carve_size<long long>(pl.bt_counts / STILE + 4) + carve_size<BtDesc>(Q);
        CKS(grow(h, h->bt, bytes));
        Carver cb(h->bt.p);
        pl.bt_rp_all = cb.take<int>(pl.bt_counts + 1);
        pl.bt_cur = cb.take<int>(pl.bt_counts + 1);
        pl.bt_ci = cb.take<int>(pl.bt_nnz);
        pl.bt_v = cb.take<char>((size_t)pl.bt_nnz * in_bytes(sr));
        pl.bt_tb = cb.take<long long>(pl.bt_counts / STILE + 4);
        pl.bt_tab = cb.take<BtDesc>(Q);
        int q = 0;
        for (int p = 0; p < P; ++p) {
            if (!want_bt(in[p])) continue;
            dp[p].bt_rp = pl.bt_rp_all + pl.bd[q].co;
            dp[p].bt_ci = pl.bt_ci;
            dp[p].bt_v = in_bytes(sr) && pl.bd[q].v ? pl.bt_v : nullptr;   // none for a pattern B
            ++q;
        }
    }

    // ---- temporary output: mask-sized for plain masks (complemented room is
    // known only after the bound scan); the gradient form writes in place
    if (pl.aligned) {
        pl.L.tmp.ci = nullptr;
        pl.L.tmp.v = in[0].aligned_out;   // one product in gradient form
    } else if (!pl.any_comp && !two_phase) {
        const int ob = out_bytes(sr);
        CKS(grow(h, h->tmp, carve_size<int>(pl.tmpn) + carve_size<char>((size_t)pl.tmpn * ob)));
        Carver ct(h->tmp.p);
        pl.L.tmp.ci = ct.take<int>(pl.tmpn);
        pl.L.tmp.v = ct.take<char>((size_t)pl.tmpn * ob);
    }

    // ---- tile index of B for every tiled product, within the memory budget;
    // products left without one walk their tiles with per-entry cursors
    pl.L.aligned = pl.aligned ? 1 : 0;
    pl.L.hash_kicks = h->hash_kicks;
    pl.nts.assign(P, 0);
    pl.tpos.assign(P, nullptr);
    if (any_tiled) {
        const int T = pl.pol.tileT[0];
        long long need = 0;
        for (int p = 0; p < P; ++p) {
            if (dp[p].n <= T) continue;
            pl.nts[p] = (dp[p].n + T - 1) / T;
            need += (long long)carve_size<int>((size_t)in[p].B->nrows * pl.nts[p] * 2);
        }
        if (h->tile_index && need <= h->tile_index_budget) {
            CKS(grow(h, h->tix, (size_t)need + 256));
            Carver ct(h->tix.p);
            for (int p = 0; p < P; ++p) {
                if (!pl.nts[p]) continue;
                pl.tpos[p] = ct.take<int>((size_t)in[p].B->nrows * pl.nts[p] * 2);
                dp[p].tpos = pl.tpos[p];
                dp[p].tstride = in[p].B->nrows;   // tile-major planes
            }
        } else {
            pl.nts.assign(P, 0);
            CKS(grow(h, h->cur, carve_size<int4>(std::max<long long>(pl.nnzA, 1))));
            pl.L.cursors = static_cast<int4 *>(h->cur.p);
        }
    }

    // ---- int64 tiled kinds: a high-word array per resident CTA (one CTA per
    // SM: their slab takes the SM's shared memory), zeroed by every call
    if (sr == MSGEMM_PLUS_TIMES_I64) {
        const size_t bytes = (size_t)h->nsm * pl.pol.tileT[0] * sizeof(unsigned);
        CKS(grow(h, h->thi, bytes));
        pl.L.tile_hi = static_cast<unsigned *>(h->thi.p);
        pl.L.tile_hi_slots = h->nsm;
        pl.thi_bytes = bytes;
    }

    // ---- MSA_G piece tables: sized by the row cap (binning assigns at most
    // Policy.grid_cap rows to the kind), so no host synchronisation is needed
    {
        bool plain_wide = false;
        for (int p = 0; p < P; ++p) plain_wide |= !in[p].comp && dp[p].n > pl.pol.tileT[0];
        pl.pol.grid_cap = 0;
        if (plain_wide && pl.pol.grid > 0) {
            const int cap = (int)std::max<long long>(GRID_CAP_MIN, std::min<long long>(GRID_CAP_MAX,
                                                                        GRID_TABLE_SLOTS / std::max(pl.gnt, 1)));
            const size_t slots = (size_t)cap * pl.gnt;
            CKS(grow(h, h->gpbuf, carve_size<int>(slots) * 2 + carve_size<int>(cap)));
            Carver cg(h->gpbuf.p);
            pl.L.g[0].cnt = cg.take<int>(slots);
            pl.L.g[0].off = cg.take<int>(slots);
            pl.L.g[0].done = cg.take<int>(cap);
            pl.gp_done_bytes = sizeof(int) * (size_t)cap;
            pl.pol.grid_cap = cap;
        }
    }

    // ---- accumulator kinds to launch (the heap kinds only when the policy
    // can pick them: forced, or in a class's preference list)
    bool any_plain = false;
    for (int p = 0; p < P; ++p) any_plain |= !in[p].comp;
    auto uses = [&](int fam) {
        if (h->force == fam) return true;
        for (int c = 0; c < NCLASS; ++c)
            for (int x = 0; x < 4 && pl.pol.pref[c][x] != F_AUTO; ++x)
                if (pl.pol.pref[c][x] == fam) return h->force == F_AUTO;
        return false;
    };
    if (any_plain) {
        if (pl.pol.slab[K_MSA_W]) pl.kinds.push_back(K_MSA_W);
        pl.kinds.insert(pl.kinds.end(), {K_HASH_W, K_MCA_W, K_HASH_B, K_HASH_L, K_MCA_B});
        if (pl.pol.q_flops_max > 0) pl.kinds.push_back(K_MCA_Q);
        if (!pl.bd.empty() ||
            std::any_of(in.begin(), in.end(), [](const ProdIn &x) { return x.bt_rp != nullptr; }))
        {
            pl.kinds.insert(pl.kinds.end(), {K_DOT_W, K_DOT_B});
            if (pl.pol.q_flops_max > 0) pl.kinds.push_back(K_DOT_Q);
        }
        if (uses(F_HEAP)) pl.kinds.push_back(K_HEAP_W);
        if (uses(F_HEAPDOT)) pl.kinds.push_back(K_HEAPDOT_W);
        pl.kinds.push_back(K_MSA_T);
        if (pl.L.g[0].cnt) pl.kinds.push_back(K_MSA_G);
    }
    if (pl.any_comp) {
        pl.kinds.insert(pl.kinds.end(), {K_CHASH_W, K_CHASH_B, K_CMSA_T});
        if (pl.pol.grid > 0) pl.kinds.push_back(K_CMSA_G);
        if (h->force == F_HEAP || h->force == F_HEAPDOT) pl.kinds.push_back(K_CHEAP_W);
    }

    // ---- products table
    pl.ps.P = P;
    pl.ps.by_value = (P == 1 && by_value) ? 1 : 0;
    pl.ps.tab = pl.dtab;
    if (pl.ps.by_value) pl.ps.p0 = dp[0];
    return MSGEMM_OK;
}

// Host -> device tables (pageable sources: never inside a capture).
msgemm_status plan_upload(msgemm_handle *h, Plan &pl) {
    cudaStream_t st = h->stream;
    if (pl.P) CK(cudaMemcpyAsync(pl.dtab, h->hprods.data(), sizeof(DevProd) * pl.P, cudaMemcpyHostToDevice, st));
    if (!pl.bd.empty())
        CK(cudaMemcpyAsync(pl.bt_tab, pl.bd.data(), sizeof(BtDesc) * pl.bd.size(), cudaMemcpyHostToDevice, st));
    return MSGEMM_OK;
}

// Device sequence, front: counters, B^T row pointers, binning.
msgemm_status seq_front(msgemm_handle *h, Plan &pl) {
    cudaStream_t st = h->stream;
    CK(cudaMemsetAsync(pl.zero_begin, 0, pl.zero_bytes, st));
    if (pl.thi_bytes) CK(cudaMemsetAsync(pl.L.tile_hi, 0, pl.thi_bytes, st));
    if (pl.gp_done_bytes) CK(cudaMemsetAsync(pl.L.g[0].done, 0, pl.gp_done_bytes, st));
    if (!pl.bd.empty()) {
        PScope ph(h, "bt_counts");
        CK(launch_bt_counts_multi(pl.bt_tab, (int)pl.bd.size(), pl.bt_nnz, pl.bt_cur, pl.bt_counts, st, h->nsm));
        CK(launch_excl_scan_int(pl.bt_cur, pl.bt_counts, pl.bt_rp_all, pl.bt_tb, st, h->nsm));
    }
    PScope ph(h, "bin");
    switch (pl.sr) {
    case MSGEMM_PLUS_TIMES_F32: CK(launch_bin_score_f32(pl.ps, pl.L.ra, pl.pol, pl.room, st, h->nsm)); break;
    case MSGEMM_PLUS_TIMES_I64: CK(launch_bin_score_i64(pl.ps, pl.L.ra, pl.pol, pl.room, st, h->nsm)); break;
    default: CK(launch_bin_score_pp(pl.ps, pl.L.ra, pl.pol, pl.room, st, h->nsm)); break;
    }
    CK(launch_bin_scatter(pl.L.ra, st, h->nsm));
    return MSGEMM_OK;
}

// Complemented products: temporary room from the per-row bounds (synchronises).
msgemm_status comp_room(msgemm_handle *h, Plan &pl) {
    cudaStream_t st = h->stream;
    long long comp_total = 0;
    int ng = 0;
    {
        PScope ph(h, "room");
        CK(launch_scan_room(pl.L.ra, pl.room, pl.tmpn, pl.room_tiles, pl.L.ra.bound_total, st, h->nsm));
        CK(cudaMemcpyAsync(&comp_total, pl.L.ra.bound_total, sizeof comp_total, cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(&ng, pl.L.ra.kind_count + K_CMSA_G, sizeof ng, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    if (ng > 0) {
        // per (row, tile) piece counts and offsets, per-row completed items
        const size_t slots = (size_t)ng * pl.gnt;
        CKS(grow(h, h->gbuf, carve_size<int>(slots) * 2 + carve_size<int>(ng)));
        Carver cg(h->gbuf.p);
        pl.L.g[1].cnt = cg.take<int>(slots);
        pl.L.g[1].off = cg.take<int>(slots);
        pl.L.g[1].done = cg.take<int>(ng);
        CK(cudaMemsetAsync(pl.L.g[1].done, 0, sizeof(int) * (size_t)ng, st));
    }
    const long long tmp_entries = pl.tmpn + comp_total;
    const int ob = out_bytes(pl.sr);
    CKS(grow(h, h->tmp, carve_size<int>(tmp_entries) + carve_size<char>((size_t)tmp_entries * ob)));
    Carver ct(h->tmp.p);
    pl.L.tmp.ci = ct.take<int>(tmp_entries);
    pl.L.tmp.v = ct.take<char>((size_t)tmp_entries * ob);
    return MSGEMM_OK;
}

// Device sequence, middle: B^T entries, tile index, one persistent kernel per
// kind, per-tile output counts.
msgemm_status seq_rows_prep(msgemm_handle *h, Plan &pl) {
    cudaStream_t st = h->stream;
    const RowArrays &ra = pl.L.ra;
    if (!pl.bd.empty()) {
        PScope ph(h, "bt_fill");
        CK(cudaMemcpyAsync(pl.bt_cur, pl.bt_rp_all, sizeof(int) * (size_t)(pl.bt_counts + 1), cudaMemcpyDeviceToDevice,
                           st));
        CK(launch_bt_fill_multi(pl.bt_tab, (int)pl.bd.size(), pl.bt_rows, in_bytes(pl.sr), pl.bt_cur, pl.bt_ci,
                                pl.bt_v, ra.any_dot, st, h->nsm));
    }
    if (std::any_of(pl.nts.begin(), pl.nts.end(), [](int x) { return x > 0; })) {
        PScope ph(h, "tile_index");
        const std::vector<DevProd> &dp = h->hprods;
        for (int p = 0; p < pl.P; ++p) {
            if (!pl.nts[p]) continue;
            // skipped on the device unless binning put rows in a tiled kind
            CK(launch_tile_bounds(dp[p].b_rp, dp[p].b_ci, dp[p].k, pl.pol.tileT[0], pl.nts[p], pl.tpos[p],
                                  ra.kind_count, st, h->nsm));
        }
    }
    return MSGEMM_OK;
}

// One persistent kernel per kind, in the instantiation of semiring sr (the
// two-phase symbolic launch passes plus-pair); heavy buckets sorted first.
msgemm_status launch_kinds(msgemm_handle *h, Plan &pl, RowLaunch L, msgemm_semiring sr, bool sort) {
    cudaStream_t st = h->stream;
    for (int kd : pl.kinds) {
        if (sort && (kd == K_MSA_T || kd == K_CMSA_T || kd == K_CMSA_G || kd == K_MSA_G)) {
            PScope ph(h, "sort_heavy");
            CK(launch_sort_heavy(pl.L.ra, kd, st));
        }
        PScope ph(h, kind_name(kd));
        L.slab = pl.pol.slab[kd];
        L.tileT = pl.pol.tileT[(kd == K_CMSA_T || kd == K_CMSA_G) ? 1 : 0];
        switch (sr) {
        case MSGEMM_PLUS_TIMES_F32: CK(launch_kind_f32(kd, pl.ps, L, st, h->nsm)); break;
        case MSGEMM_PLUS_TIMES_I64: CK(launch_kind_i64(kd, pl.ps, L, st, h->nsm)); break;
        default: CK(launch_kind_pp(kd, pl.ps, L, st, h->nsm)); break;
        }
    }
    return MSGEMM_OK;
}

msgemm_status seq_middle(msgemm_handle *h, Plan &pl) {
    cudaStream_t st = h->stream;
    const RowArrays &ra = pl.L.ra;
    CKS(seq_rows_prep(h, pl));
    CKS(launch_kinds(h, pl, pl.L, pl.sr, true));
    if (pl.aligned) return MSGEMM_OK;
    PScope ph(h, "count");
    CK(launch_count_tiles(pl.ps, ra, pl.ntiles, pl.tile_sums, pl.tile_offs, pl.prod_tot, pl.chunk_start, st, h->nsm));
    return MSGEMM_OK;
}

// Complemented products: exact output sizes (synchronises), outputs allocated.
msgemm_status comp_outputs(msgemm_handle *h, std::vector<ProdIn> &in, Plan &pl, bool all = false) {
    cudaStream_t st = h->stream;
    const int P = pl.P;
    std::vector<DevProd> &dp = h->hprods;
    std::vector<long long> tot(P);
    CK(cudaMemcpyAsync(tot.data(), pl.prod_tot + P, sizeof(long long) * P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const int ob = out_bytes(pl.sr);
    std::vector<int> who;
    std::vector<size_t> ci_sz, v_sz;
    for (int p = 0; p < P; ++p) {
        if (!in[p].comp && !all) continue;
        if (tot[p] >= (1LL << 31)) return fail(h, MSGEMM_ERR_OVERFLOW, "product %d has >= 2^31 entries", p);
        who.push_back(p);
        ci_sz.push_back(sizeof(int) * (size_t)tot[p]);
        v_sz.push_back((size_t)ob * (size_t)tot[p]);
    }
    // one allocation for the columns of all these products, one for the values
    const std::vector<char *> ci = carve_alloc(h, ci_sz), v = carve_alloc(h, v_sz);
    for (size_t x = 0; x < who.size(); ++x) {
        const int p = who[x];
        msgemm_csr_out *C = in[p].C;
        if (!ci[x] || !v[x]) return fail(h, MSGEMM_ERR_OOM, "output allocation failed");
        C->capacity = tot[p];
        C->colidx = reinterpret_cast<int32_t *>(ci[x]);
        C->values = v[x];
        dp[p].c_ci = C->colidx;
        dp[p].c_v = C->values;
        pl.cap += tot[p];
    }
    if (pl.ps.by_value) pl.ps.p0 = dp[0];
    CK(cudaMemcpyAsync(pl.dtab, dp.data(), sizeof(DevProd) * P, cudaMemcpyHostToDevice, st));
    return MSGEMM_OK;
}

// Device sequence, back: chunked compaction into C.
msgemm_status seq_compact(msgemm_handle *h, Plan &pl) {
    PScope ph(h, "compact");
    // chunks: at most one per tile plus one per CCH entries of the capacity
    CK(launch_compact(pl.ps, pl.L.ra, pl.L.tmp, pl.ntiles, pl.tile_offs, pl.chunk_start,
                      pl.ntiles + pl.cap / CCH + 1, out_bytes(pl.sr), h->stream, h->nsm));
    return MSGEMM_OK;
}

template <class T> void key_put(std::string &k, const T &x) {
    k.append(reinterpret_cast<const char *>(&x), sizeof x);
}

// Everything a captured sequence bakes in: policy, launch arguments,
// workspace and input pointers and sizes (not the outputs, which the device
// table carries and which are uploaded before every replay).
std::string graph_key(const msgemm_handle *h, const Plan &pl) {
    std::string k;
    key_put(k, pl.sr);
    key_put(k, pl.P);
    key_put(k, pl.pol);
    key_put(k, pl.L);
    key_put(k, pl.ps.tab);
    key_put(k, pl.R);
    key_put(k, pl.ntiles);
    key_put(k, pl.cap);
    key_put(k, pl.zero_begin);
    key_put(k, pl.zero_bytes);
    key_put(k, h->nsm);
    for (int kd : pl.kinds) key_put(k, kd);
    for (const BtDesc &b : pl.bd) key_put(k, b);
    key_put(k, pl.bt_rp_all);
    key_put(k, pl.bt_tab);
    for (int p = 0; p < pl.P; ++p) {
        const DevProd &d = h->hprods[p];
        for (const void *ptr : {(const void *)d.m_rp, (const void *)d.m_ci, (const void *)d.a_rp, (const void *)d.a_ci,
                                d.a_v, (const void *)d.b_rp, (const void *)d.b_ci, d.b_v, (const void *)d.bt_rp,
                                (const void *)d.bt_ci, d.bt_v, (const void *)d.tpos})
            key_put(k, ptr);
        for (long long x : {(long long)d.m, (long long)d.n, (long long)d.k, (long long)d.complement,
                            (long long)d.a_sorted, d.row0, d.tile0, d.abase, d.tmp0, (long long)d.tstride,
                            (long long)pl.nts[p]})
            key_put(k, x);
    }
    return k;
}

// Replays the cached graph of this plan, or captures a new one (on the
// handle's private capture stream: nothing runs during the capture) and
// launches it on the handle's stream.
msgemm_status run_graph(msgemm_handle *h, Plan &pl) {
    std::string key = graph_key(h, pl);
    if (h->gexec && key == h->gkey) {
        CK(cudaGraphLaunch(h->gexec, h->stream));
        g_kernel_launches.fetch_add(h->gkernels, std::memory_order_relaxed);
        return MSGEMM_OK;
    }
    if (h->gexec) {
        cudaGraphExecDestroy(h->gexec);
        h->gexec = nullptr;
        h->gkey.clear();
    }
    if (!h->cap_stream) CK(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const long long before = g_kernel_launches.load();
    cudaStream_t user = h->stream;
    h->stream = h->cap_stream;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    msgemm_status rs = MSGEMM_OK;
    if (e == cudaSuccess) {
        rs = seq_front(h, pl);
        if (rs == MSGEMM_OK) rs = seq_middle(h, pl);
        if (rs == MSGEMM_OK) rs = seq_compact(h, pl);
    }
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamEndCapture(h->cap_stream, &g);
    h->stream = user;
    // launches counted during the capture were recorded, not run
    g_kernel_launches.fetch_sub(g_kernel_launches.load() - before, std::memory_order_relaxed);
    if (rs != MSGEMM_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
        return rs != MSGEMM_OK ? rs : fail(h, MSGEMM_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
    }
    size_t nn = 0;
    long long nk = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType t;
                if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++nk;
            }
    }
    e = cudaGraphInstantiate(&h->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->gexec = nullptr;
        return fail(h, MSGEMM_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
    }
    h->gkey = std::move(key);
    h->gkernels = nk;
    ++h->gcaptures;
    CK(cudaGraphLaunch(h->gexec, h->stream));
    g_kernel_launches.fetch_add(nk, std::memory_order_relaxed);
    return MSGEMM_OK;
}

// The whole one-phase pipeline for a set of products (Sec. 4-6).  With
// use_graph, plain masks, no validation and no profiling, the device
// sequence runs as a replayed CUDA graph; otherwise eagerly.
msgemm_status run_pipeline(msgemm_handle *h, std::vector<ProdIn> &in, msgemm_semiring sr, bool build_bt,
                           bool validate, bool use_graph = false) {
    bool graph = use_graph && !validate && !h->profile;
    for (const ProdIn &x : in) graph = graph && !x.comp && !x.aligned_out;
    Plan pl;
    CKS(plan_prepare(h, in, sr, build_bt, !graph, pl));
    CKS(plan_upload(h, pl));
    // optional input validation: synchronises, and rejects invalid input
    // before any kernel that would index through it runs
    if (validate) {
        PScope ph(h, "validate");
        std::vector<const msgemm_csr *> mats;
        for (const ProdIn &x : in) mats.insert(mats.end(), {x.M, x.A, x.B});
        CKS(validate_inputs(h, mats));
    }
    if (graph) return run_graph(h, pl);
    CKS(seq_front(h, pl));
    if (pl.any_comp) CKS(comp_room(h, pl));
    CKS(seq_middle(h, pl));
    if (pl.aligned) return MSGEMM_OK;
    if (pl.any_comp) CKS(comp_outputs(h, in, pl));
    return seq_compact(h, pl);
}

// Sec. 6, two-phase form.  Symbolic: every kind runs in its plus-pair
// instantiation (indices only; its per-row state is never larger than the
// other semirings', so the binning's choices fit) and counts each row's
// entries without writing any.  The counts give C's row pointers; C is then
// allocated to its exact size (synchronises).  Numeric: every kind runs again
// in the call's semiring and writes each row straight to its final place.
// No temporary output and no compaction; the (row, tile) grid kinds are not
// used (their pieces need a temporary's room), nor the CUDA graph.
msgemm_status run_two_phase(msgemm_handle *h, std::vector<ProdIn> &in, msgemm_semiring sr, bool build_bt,
                            bool validate) {
    Plan pl;
    CKS(plan_prepare(h, in, sr, build_bt, true, pl, true));
    CKS(plan_upload(h, pl));
    if (validate) {
        PScope ph(h, "validate");
        std::vector<const msgemm_csr *> mats;
        for (const ProdIn &x : in) mats.insert(mats.end(), {x.M, x.A, x.B});
        CKS(validate_inputs(h, mats));
    }
    cudaStream_t st = h->stream;
    CKS(seq_front(h, pl));
    CKS(seq_rows_prep(h, pl));
    RowLaunch L = pl.L;
    L.count_only = 1;
    {
        PScope ph(h, "symbolic");
        CKS(launch_kinds(h, pl, L, MSGEMM_PLUS_PAIR_I64, true));
        CK(launch_count_tiles(pl.ps, pl.L.ra, pl.ntiles, pl.tile_sums, pl.tile_offs, pl.prod_tot, pl.chunk_start, st,
                              h->nsm));
    }
    CKS(comp_outputs(h, in, pl, true));
    {
        PScope ph(h, "row_offsets");
        CK(launch_row_offsets(pl.ps, pl.L.ra, pl.ntiles, pl.tile_offs, st, h->nsm));
        CK(cudaMemsetAsync(pl.L.ra.kind_next, 0, sizeof(int) * NKIND, st));
    }
    L = pl.L;
    L.direct = 1;
    PScope ph(h, "numeric");
    return launch_kinds(h, pl, L, sr, false);
}

// One-phase or two-phase, by the handle's option.
msgemm_status run_products(msgemm_handle *h, std::vector<ProdIn> &in, msgemm_semiring sr, bool validate,
                           bool use_graph) {
    if (h->phases == 2) return run_two_phase(h, in, sr, true, validate);
    return run_pipeline(h, in, sr, true, validate, use_graph);
}

// Outputs of n products: row pointers and entry counts, and for products
// sized by their mask (no_room[p] == 0: plain, one phase) columns and values
// of the mask's size; the rest get columns and values once their exact size
// is known.  One allocation per array kind for all n products.
msgemm_status alloc_outs(msgemm_handle *h, int n, const msgemm_csr *M, const int *no_room, msgemm_semiring sr,
                         msgemm_csr_out *C) {
    std::vector<size_t> rp_sz(n), nz_sz(n, sizeof(int64_t)), ci_sz, v_sz;
    for (int p = 0; p < n; ++p) {
        memset(&C[p], 0, sizeof C[p]);
        C[p].nrows = M[p].nrows;
        C[p].ncols = M[p].ncols;
        rp_sz[p] = sizeof(int) * ((size_t)M[p].nrows + 1);
        if (!no_room[p]) {
            ci_sz.push_back(sizeof(int) * (size_t)M[p].nnz);
            v_sz.push_back((size_t)out_bytes(sr) * (size_t)M[p].nnz);
        }
    }
    const std::vector<char *> rp = carve_alloc(h, rp_sz), nz = carve_alloc(h, nz_sz);
    const std::vector<char *> ci = carve_alloc(h, ci_sz), v = carve_alloc(h, v_sz);
    size_t x = 0;
    for (int p = 0; p < n; ++p) {
        C[p].rowptr = reinterpret_cast<int32_t *>(rp[p]);
        C[p].d_nnz = reinterpret_cast<int64_t *>(nz[p]);
        if (!C[p].rowptr || !C[p].d_nnz) return fail(h, MSGEMM_ERR_OOM, "output allocation failed");
        if (!no_room[p]) {
            C[p].capacity = M[p].nnz;
            C[p].colidx = reinterpret_cast<int32_t *>(ci[x]);
            C[p].values = v[x];
            ++x;
            if (!C[p].colidx || !C[p].values) return fail(h, MSGEMM_ERR_OOM, "output allocation failed");
        }
    }
    return MSGEMM_OK;
}

msgemm_status alloc_out(msgemm_handle *h, const msgemm_csr *M, int comp, msgemm_semiring sr, msgemm_csr_out *C) {
    return alloc_outs(h, 1, M, &comp, sr, C);
}

msgemm_status check_product(msgemm_handle *h, const msgemm_csr *M, const msgemm_csr *A, const msgemm_csr *B,
                            msgemm_semiring sr) {
    if (sr < MSGEMM_PLUS_TIMES_F32 || sr > MSGEMM_PLUS_PAIR_I64) return fail(h, MSGEMM_ERR_INVALID, "unknown semiring");
    // values may be NULL: plus-pair never reads them, and under plus-times a
    // NULL value array makes A or B a pattern operand (every stored value 1)
    CKS(check_csr(h, M, "M", false));
    CKS(check_csr(h, A, "A", false));
    CKS(check_csr(h, B, "B", false));
    if (M->nrows != A->nrows || A->ncols != B->nrows || M->ncols != B->ncols)
        return fail(h, MSGEMM_ERR_SHAPE, "shapes do not chain: M %dx%d, A %dx%d, B %dx%d", M->nrows, M->ncols, A->nrows,
                    A->ncols, B->nrows, B->ncols);
    return MSGEMM_OK;
}

// ---- autotuning (msgemm_autotune): the policy knobs the binning pass reads
struct Tuned {
    int warp_flops_max = 65536;
    float dot_ratio = 2.0f;
    int warp_slab = 4608;
    long long grid_min_flops = 1LL << 20;
    unsigned char pref[NCLASS][4];
    int q_flops_max = 1024;
    int hash_slab = 4608;
};

Tuned current_tuned(const msgemm_handle *h) {
    Tuned t;
    t.warp_flops_max = h->warp_flops_max;
    t.dot_ratio = h->dot_ratio;
    t.warp_slab = h->warp_slab;
    t.grid_min_flops = h->grid_min_flops;
    memcpy(t.pref, h->pref, sizeof t.pref);
    t.q_flops_max = h->q_flops_max;
    t.hash_slab = h->hash_slab;
    return t;
}

void apply_tuned(msgemm_handle *h, const Tuned &t) {
    h->warp_flops_max = t.warp_flops_max;
    h->dot_ratio = t.dot_ratio;
    h->warp_slab = t.warp_slab;
    h->grid_min_flops = t.grid_min_flops;
    memcpy(h->pref, t.pref, sizeof t.pref);
    h->q_flops_max = t.q_flops_max;
    h->hash_slab = t.hash_slab;
}

// Cache file: a JSON object, one entry per line,
//   "<device name>|<semiring>": {"warp_flops_max": W, "dot_ratio": D, "warp_slab": S, "grid_min_flops": G,
//                                "pref": [[f,f,f,f], ...], "q_flops_max": Q, "hash_slab": S2}
// with NCLASS preference rows of accumulator families (msgemm_accumulator);
// an entry without q_flops_max or hash_slab (written before they existed)
// keeps their defaults.
void read_tuned(const char *path, std::map<std::string, Tuned> &out) {
    FILE *f = fopen(path, "r");
    if (!f) return;
    char line[4096];
    while (fgets(line, sizeof line, f)) {
        const char *q0 = strchr(line, '"');
        if (!q0) continue;
        const char *q1 = strstr(q0 + 1, "\":");
        if (!q1) continue;
        std::string key(q0 + 1, q1);
        std::vector<double> num;
        for (const char *c = q1 + 2; *c;) {
            if ((*c >= '0' && *c <= '9') || *c == '-' || *c == '.') {
                char *e = nullptr;
                num.push_back(strtod(c, &e));
                c = e;
            } else {
                ++c;
            }
        }
        if (num.size() < 4 + NCLASS * 4 || num.size() > 6 + NCLASS * 4) continue;
        Tuned t;
        if (num[0] < 0 || num[0] > 1e9 || !(num[1] > 0) || num[1] > 1e6) continue;
        if (num[2] < 1024 || num[2] > 24576 || (int)num[2] % 16) continue;
        t.warp_flops_max = (int)num[0];
        t.dot_ratio = (float)num[1];
        t.warp_slab = (int)num[2];
        if (num[3] < 0 || num[3] > 9.3e18) continue;
        t.grid_min_flops = (long long)num[3];
        bool ok = true;
        for (int c = 0; c < NCLASS; ++c)
            for (int x = 0; x < 4; ++x) {
                const double v = num[4 + c * 4 + x];
                ok &= v >= F_AUTO && v <= F_HEAPDOT && v == (int)v;
                t.pref[c][x] = (unsigned char)v;
            }
        if (num.size() >= 5 + NCLASS * 4) {
            const double q = num[4 + NCLASS * 4];
            ok &= q >= 0 && q <= (1 << 20) && q == (int)q;
            t.q_flops_max = (int)q;
        }
        if (num.size() == 6 + NCLASS * 4) {
            const double s = num[5 + NCLASS * 4];
            ok &= s >= 1024 && s <= 24576 && s == (int)s && (int)s % 16 == 0;
            t.hash_slab = (int)s;
        }
        if (ok) out[key] = t;
    }
    fclose(f);
}

bool write_tuned(const char *path, const std::map<std::string, Tuned> &m) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : m) {
        const Tuned &t = kv.second;
        fprintf(f, "\"%s\": {\"warp_flops_max\": %d, \"dot_ratio\": %g, \"warp_slab\": %d, \"grid_min_flops\": %lld, \"pref\": [",
                kv.first.c_str(), t.warp_flops_max, (double)t.dot_ratio, t.warp_slab, t.grid_min_flops);
        for (int c = 0; c < NCLASS; ++c)
            fprintf(f, "%s[%d, %d, %d, %d]", c ? ", " : "", t.pref[c][0], t.pref[c][1], t.pref[c][2], t.pref[c][3]);
        fprintf(f, "], \"q_flops_max\": %d, \"hash_slab\": %d}%s\n", t.q_flops_max, t.hash_slab, ++i < m.size() ? "," : "");
    }
    fprintf(f, "}\n");
    const bool ok = fclose(f) == 0;
    return ok && rename(tmp.c_str(), path) == 0;
}

// Coordinate search over the policy, timing the whole given batch: first the
// accumulator family tried first for each row class that carries work (the
// classes by descending work), then the warp/CTA split and the pull ratio.
// Every candidate computes the same result; only time differs.
struct Tuner {
    msgemm_handle *h;
    int P;
    const msgemm_csr *M, *A, *B;
    const int *comp;
    msgemm_semiring sr;
    cudaEvent_t ea = nullptr, eb = nullptr;
    Tuner(msgemm_handle *h_, int P_, const msgemm_csr *M_, const int *c_, const msgemm_csr *A_, const msgemm_csr *B_,
          msgemm_semiring sr_)
        : h(h_), P(P_), M(M_), A(A_), B(B_), comp(c_), sr(sr_) {}
    ~Tuner() {
        if (ea) cudaEventDestroy(ea);
        if (eb) cudaEventDestroy(eb);
    }

    msgemm_status run_once(float *ms) {
        std::vector<msgemm_csr_out> C(P);
        std::vector<ProdIn> in(P);
        std::vector<int> no_room(P);
        h->out_allocs.clear();
        for (int p = 0; p < P; ++p) {
            const int c = comp ? comp[p] != 0 : 0;
            no_room[p] = c || h->phases == 2;
            in[p].M = &M[p]; in[p].A = &A[p]; in[p].B = &B[p]; in[p].comp = c; in[p].C = &C[p];
        }
        msgemm_status rs = alloc_outs(h, P, M, no_room.data(), sr, C.data());
        if (rs == MSGEMM_OK && cudaEventRecord(ea, h->stream) != cudaSuccess) rs = MSGEMM_ERR_CUDA;
        if (rs == MSGEMM_OK) rs = run_products(h, in, sr, false, false);
        if (rs == MSGEMM_OK && cudaEventRecord(eb, h->stream) != cudaSuccess) rs = MSGEMM_ERR_CUDA;
        if (rs == MSGEMM_OK && (cudaEventSynchronize(eb) != cudaSuccess || cudaEventElapsedTime(ms, ea, eb) != cudaSuccess))
            rs = fail(h, MSGEMM_ERR_CUDA, "autotune timing failed");
        cudaStreamSynchronize(h->stream);
        for (void *ptr : h->out_allocs) dev_free(h, ptr);
        h->out_allocs.clear();
        return rs;
    }

    // median of three timed runs after one untimed
    msgemm_status measure(float *ms) {
        float t[3], w;
        CKS(run_once(&w));
        for (float &x : t) CKS(run_once(&x));
        std::sort(t, t + 3);
        *ms = t[1];
        return MSGEMM_OK;
    }

    // work per row class (sum of push flops) from the last run's binning
    msgemm_status class_work(std::vector<double> &work) {
        work.assign(NCLASS, 0.0);
        const long long R = h->last_R;
        if (R == 0) return MSGEMM_OK;
        std::vector<long long> flops(R);
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaMemcpy(flops.data(), h->rows.p, sizeof(long long) * R, cudaMemcpyDeviceToHost));   // ra.flops
        long long r = 0;
        for (int p = 0; p < P; ++p) {
            std::vector<int> rp(M[p].nrows + 1);
            CK(cudaMemcpy(rp.data(), M[p].rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost));
            for (int i = 0; i < M[p].nrows; ++i, ++r)
                if (!(comp && comp[p])) work[row_class(flops[r], rp[i + 1] - rp[i])] += (double)flops[r];
        }
        return MSGEMM_OK;
    }

    msgemm_status tune() {
        CK(cudaEventCreate(&ea));
        CK(cudaEventCreate(&eb));
        float best;
        CKS(measure(&best));
        const Tuned start = current_tuned(h);
        const float best_start = best;
        // The class lists are searched with pull off, so that the rows pull
        // would take meet every family too; pull comes back in the ratio
        // search at the end, and the start wins if nothing beats it.
        if (h->allow_dot) {
            h->dot_ratio = 1e6f;
            CKS(measure(&best));
        }
        std::vector<double> work;
        CKS(class_work(work));
        double total = 0;
        for (double w : work) total += w;
        std::vector<int> order;
        for (int c = 0; c < NCLASS; ++c)
            if (work[c] > 0.005 * total) order.push_back(c);
        std::sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
        const float keep = 0.98f;   // a candidate must win by 2% to replace the incumbent
        for (int c : order) {
            unsigned char base[4];
            memcpy(base, h->pref[c], 4);
            unsigned char best_pref[4];
            memcpy(best_pref, base, 4);
            for (int fam : {F_MSA, F_HASH, F_MCA, F_HEAP, F_HEAPDOT}) {
                if (base[0] == fam) continue;
                unsigned char cand[4] = {(unsigned char)fam, 0, 0, 0};
                int n = 1;
                for (int x = 0; x < 4 && base[x] != F_AUTO; ++x)
                    if (base[x] != fam && n < 4) cand[n++] = base[x];
                while (n < 4) cand[n++] = F_AUTO;
                memcpy(h->pref[c], cand, 4);
                float t;
                CKS(measure(&t));
                if (t < best * keep) {
                    best = t;
                    memcpy(best_pref, cand, 4);
                }
            }
            memcpy(h->pref[c], best_pref, 4);
        }
        const int wbest0 = h->warp_flops_max;
        int wbest = wbest0;
        for (int w : {8192, 16384, 32768, 65536, 131072, 262144}) {
            if (w == wbest0) continue;
            h->warp_flops_max = w;
            float t;
            CKS(measure(&t));
            if (t < best * keep) { best = t; wbest = w; }
        }
        h->warp_flops_max = wbest;
        const int qbest0 = h->q_flops_max;
        int qbest = qbest0;
        for (int q : {0, 256, 1024, 4096, 16384, 65536, 1 << 20}) {
            if (q == qbest0) continue;
            h->q_flops_max = q;
            float t;
            CKS(measure(&t));
            if (t < best * keep) { best = t; qbest = q; }
        }
        h->q_flops_max = qbest;
        const int sbest0 = h->warp_slab;
        int sbest = sbest0;
        for (int sl : {3072, 3584, 4096, 4608, 6144, 9216}) {
            if (sl == sbest0) continue;
            h->warp_slab = sl;
            float t;
            CKS(measure(&t));
            if (t < best * keep) { best = t; sbest = sl; }
        }
        h->warp_slab = sbest;
        const int hbest0 = h->hash_slab;
        int hbest = hbest0;
        for (int sl : {3072, 4608, 6144, 9216, 12288}) {
            if (sl == hbest0) continue;
            h->hash_slab = sl;
            float t;
            CKS(measure(&t));
            if (t < best * keep) { best = t; hbest = sl; }
        }
        h->hash_slab = hbest;
        const long long gbest0 = h->grid_min_flops;
        long long gbest = gbest0;
        for (long long g : {1LL << 18, 1LL << 19, 1LL << 20, 1LL << 21, 1LL << 22, 1LL << 62}) {
            if (g == gbest0) continue;
            h->grid_min_flops = g;
            float t;
            CKS(measure(&t));
            if (t < best * keep) { best = t; gbest = g; }
        }
        h->grid_min_flops = gbest;
        if (h->allow_dot) {
            const float dbest0 = h->dot_ratio;
            float dbest = dbest0;
            for (float d : {0.5f, 1.0f, 2.0f, 4.0f, 8.0f}) {
                if (d == dbest0) continue;
                h->dot_ratio = d;
                float t;
                CKS(measure(&t));
                if (t < best * keep) { best = t; dbest = d; }
            }
            h->dot_ratio = dbest;
        }
        if (best > best_start) apply_tuned(h, start);
        return MSGEMM_OK;
    }
};

}  // namespace

// ===================================================================== C ABI
extern "C" {

msgemm_status msgemm_create(msgemm_handle **handle, void *stream, msgemm_alloc_fn alloc, msgemm_free_fn free_fn,
                            void *ctx) {
    if (!handle) return MSGEMM_ERR_INVALID;
    *handle = nullptr;
    if ((alloc == nullptr) != (free_fn == nullptr)) return MSGEMM_ERR_INVALID;
    msgemm_handle *h = new msgemm_handle();
    h->stream = static_cast<cudaStream_t>(stream);
    h->alloc = alloc;
    h->free_fn = free_fn;
    h->ctx = ctx;
    default_pref(h->pref);
    if (cudaGetDevice(&h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&h->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return MSGEMM_ERR_CUDA;
    }
    if (grow(h, h->small, 16384) != MSGEMM_OK) {
        delete h;
        return MSGEMM_ERR_OOM;
    }
    h->d_err = static_cast<unsigned *>(h->small.p);
    if (cudaMemsetAsync(h->small.p, 0, h->small.cap, h->stream) != cudaSuccess) {
        dev_free(h, h->small.p);
        delete h;
        return MSGEMM_ERR_CUDA;
    }
    *handle = h;
    return MSGEMM_OK;
}

msgemm_status msgemm_set_stream(msgemm_handle *h, void *stream) {
    if (!h) return MSGEMM_ERR_INVALID;
    if (static_cast<cudaStream_t>(stream) == h->stream) return MSGEMM_OK;
    CK(cudaStreamSynchronize(h->stream));
    h->stream = static_cast<cudaStream_t>(stream);
    return MSGEMM_OK;
}

msgemm_status msgemm_set_option(msgemm_handle *h, msgemm_option opt, int64_t value) {
    if (!h) return MSGEMM_ERR_INVALID;
    switch (opt) {
    case MSGEMM_OPT_FORCE_ACCUM:
        if (value < MSGEMM_ACC_AUTO || value > MSGEMM_ACC_HEAPDOT) return fail(h, MSGEMM_ERR_INVALID, "bad accumulator");
        h->force = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_VALIDATE: h->validate = value != 0; return MSGEMM_OK;
    case MSGEMM_OPT_DOT: h->allow_dot = value != 0; return MSGEMM_OK;
    case MSGEMM_OPT_PROFILE: h->profile = value != 0; return MSGEMM_OK;
    case MSGEMM_OPT_TILE_INDEX: h->tile_index = value != 0; return MSGEMM_OK;
    case MSGEMM_OPT_WARP_SLAB:
        if (value < 1024 || value > 24576 || value % 16) return fail(h, MSGEMM_ERR_INVALID, "warp slab bytes");
        h->warp_slab = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_HASH_SLAB:
        if (value < 1024 || value > 24576 || value % 16) return fail(h, MSGEMM_ERR_INVALID, "hash slab bytes");
        h->hash_slab = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_GRID_MIN_FLOPS:
        if (value < 0) return fail(h, MSGEMM_ERR_INVALID, "grid flop bound must be >= 0");
        h->grid_min_flops = value;
        return MSGEMM_OK;
    case MSGEMM_OPT_GRID:
        if (value < 0 || value > 2) return fail(h, MSGEMM_ERR_INVALID, "grid mode is 0, 1 or 2");
        h->grid = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_PHASES:
        if (value != 1 && value != 2) return fail(h, MSGEMM_ERR_INVALID, "phases is 1 or 2");
        h->phases = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_QTEAM_FLOPS:
        if (value < 0 || value > (1 << 20)) return fail(h, MSGEMM_ERR_INVALID, "team-of-eight flop bound is 0..2^20");
        h->q_flops_max = (int)value;
        return MSGEMM_OK;
    case MSGEMM_OPT_HASH_KICKS:
        if (value < 0 || value > 4096) return fail(h, MSGEMM_ERR_INVALID, "hash kicks is 0..4096");
        h->hash_kicks = (int)value;
        return MSGEMM_OK;
    default: return fail(h, MSGEMM_ERR_INVALID, "unknown option %d", (int)opt);
    }
}

msgemm_status msgemm_run(msgemm_handle *h, const msgemm_csr *M, int complement, const msgemm_csr *A,
                         const msgemm_csr *B, msgemm_semiring sr, msgemm_csr_out *C) {
    if (!h || !C) return fail(h, MSGEMM_ERR_INVALID, "NULL handle or output");
    h->nprof = 0;
    CKS(check_product(h, M, A, B, sr));
    const int comp = complement != 0;
    h->out_allocs.clear();
    CKS(alloc_out(h, M, comp || h->phases == 2, sr, C));
    std::vector<ProdIn> in(1);
    in[0].M = M; in[0].A = A; in[0].B = B; in[0].comp = comp; in[0].C = C;
    return run_products(h, in, sr, h->validate, false);
}

namespace {

msgemm_status check_backward(msgemm_handle *h, const msgemm_csr *A, const msgemm_csr *B, const msgemm_csr *G,
                             msgemm_semiring sr) {
    if (sr != MSGEMM_PLUS_TIMES_F32) return fail(h, MSGEMM_ERR_UNSUPPORTED, "backward is defined for plus-times fp32");
    CKS(check_csr(h, A, "A", true));
    CKS(check_csr(h, B, "B", true));
    if (G) {
        CKS(check_csr(h, G, "G", true));
        if (A->ncols != B->nrows || G->nrows != A->nrows || G->ncols != B->ncols)
            return fail(h, MSGEMM_ERR_SHAPE, "shapes do not chain: A %dx%d, B %dx%d, G %dx%d", A->nrows, A->ncols,
                        B->nrows, B->ncols, G->nrows, G->ncols);
    } else if (A->ncols != B->nrows) {
        return fail(h, MSGEMM_ERR_SHAPE, "shapes do not chain: A %dx%d, B %dx%d", A->nrows, A->ncols, B->nrows,
                    B->ncols);
    }
    return MSGEMM_OK;
}

// dA = pattern(A) .* (G B^T): mask A, left G (m x n), right B^T (n x k)
// given as Bt; the pull kernel reads columns of B^T, which are the rows of B.
msgemm_status backward_dA(msgemm_handle *h, const msgemm_csr *A, const msgemm_csr *B, const msgemm_csr *G,
                          const msgemm_csr &Bt, float *dA_vals) {
    msgemm_csr Mx = *A;
    Mx.values = nullptr;
    std::vector<ProdIn> in(1);
    in[0].M = &Mx; in[0].A = G; in[0].B = &Bt; in[0].comp = 0;
    in[0].bt_rp = B->rowptr; in[0].bt_ci = B->colidx; in[0].bt_v = B->values;
    in[0].aligned_out = dA_vals;
    CK(cudaMemsetAsync(dA_vals, 0, sizeof(float) * (size_t)A->nnz, h->stream));
    return A->nnz > 0 ? run_pipeline(h, in, MSGEMM_PLUS_TIMES_F32, false, false) : MSGEMM_OK;
}

// dB = pattern(B) .* (A^T G): mask B, left A^T (k x m) given as At, right G.
msgemm_status backward_dB(msgemm_handle *h, const msgemm_csr *B, const msgemm_csr *G, const msgemm_csr &At,
                          int at_sorted, float *dB_vals) {
    msgemm_csr Mx = *B;
    Mx.values = nullptr;
    std::vector<ProdIn> in(1);
    in[0].M = &Mx; in[0].A = &At; in[0].B = G; in[0].comp = 0;
    in[0].a_sorted = at_sorted;
    in[0].aligned_out = dB_vals;
    CK(cudaMemsetAsync(dB_vals, 0, sizeof(float) * (size_t)B->nnz, h->stream));
    return B->nnz > 0 ? run_pipeline(h, in, MSGEMM_PLUS_TIMES_F32, false, false) : MSGEMM_OK;
}

}  // namespace

msgemm_status msgemm_backward(msgemm_handle *h, const msgemm_csr *A, const msgemm_csr *B, const msgemm_csr *G,
                              msgemm_semiring sr, float *dA_vals, float *dB_vals) {
    if (!h) return MSGEMM_ERR_INVALID;
    h->nprof = 0;
    CKS(check_backward(h, A, B, G, sr));
    if (h->validate) CKS(validate_inputs(h, {A, B, G}));
    cudaStream_t st = h->stream;
    // transposes B^T (n x k) and A^T (k x m), values carried, rows unsorted
    struct T { int *rp, *cur, *ci; float *v; long long *tb; };
    auto tsize = [](const msgemm_csr *X) {
        return carve_size<int>((size_t)X->ncols + 1) * 2 + carve_size<int>(X->nnz) + carve_size<float>(X->nnz) +
               carve_size<long long>(X->ncols / STILE + 4);
    };
    Buf tb;
    tb.p = dev_alloc(h, tsize(A) + tsize(B) + 1024);
    if (!tb.p) return fail(h, MSGEMM_ERR_OOM, "transpose workspace allocation failed");
    Carver cv(tb.p);
    auto mk = [&](const msgemm_csr *X) {
        T t;
        t.rp = cv.take<int>((size_t)X->ncols + 1);
        t.cur = cv.take<int>((size_t)X->ncols + 1);
        t.ci = cv.take<int>(X->nnz);
        t.v = cv.take<float>(X->nnz);
        t.tb = cv.take<long long>(X->ncols / STILE + 4);
        return t;
    };
    T Bt = mk(B), At = mk(A);
    msgemm_status rs = MSGEMM_OK;
    // sorted: rows of the transpose in ascending column order (needed when it
    // is the right operand, whose rows the column-tiled MSA walks by cursor)
    auto transpose = [&](const msgemm_csr *X, T &t, bool sorted) -> msgemm_status {
        PScope ph(h, "transpose");
        CK(launch_col_counts(X->colidx, X->nnz, X->ncols, t.cur, st, h->nsm));
        CK(launch_excl_scan_int(t.cur, X->ncols, t.rp, t.tb, st, h->nsm));
        CK(cudaMemcpyAsync(t.cur, t.rp, sizeof(int) * ((size_t)X->ncols + 1), cudaMemcpyDeviceToDevice, st));
        CK(launch_transpose_fill(X->rowptr, X->colidx, X->values, 4, X->nrows, X->ncols, t.cur, t.ci, t.v, nullptr, st,
                                 h->nsm));
        if (sorted) CK(launch_segsort(t.rp, t.ci, t.v, 4, X->ncols, t.cur, st, h->nsm));   // cursors are free now
        return MSGEMM_OK;
    };
    if (dA_vals) {
        rs = transpose(B, Bt, true);
        if (rs == MSGEMM_OK) {
            const msgemm_csr Bx{B->ncols, B->nrows, B->nnz, Bt.rp, Bt.ci, Bt.v};
            rs = backward_dA(h, A, B, G, Bx, dA_vals);
        }
    }
    if (rs == MSGEMM_OK && dB_vals) {
        rs = transpose(A, At, false);
        if (rs == MSGEMM_OK) {
            const msgemm_csr Ax{A->ncols, A->nrows, A->nnz, At.rp, At.ci, At.v};
            rs = backward_dB(h, B, G, Ax, 0, dB_vals);
        }
    }
    // the transpose buffer is released in stream order (the callback's free
    // must honour stream order; cudaFree synchronises)
    dev_free(h, tb.p);
    return rs;
}

// Transposed patterns of a backward pass, built once (see msgemm.h).
struct msgemm_backward_plan {
    int device = 0;
    const int32_t *a_rp = nullptr, *a_ci = nullptr, *b_rp = nullptr, *b_ci = nullptr;
    int32_t am = 0, an = 0, bm = 0, bn = 0;
    int64_t annz = 0, bnnz = 0;
    void *mem = nullptr;
    int *bt_rp = nullptr, *bt_ci = nullptr, *bt_perm = nullptr;   // B^T (n x k), rows ascending
    int *at_rp = nullptr, *at_ci = nullptr, *at_perm = nullptr;   // A^T (k x m), rows ascending
    float *bt_v = nullptr, *at_v = nullptr;                       // values gathered by each call
};

msgemm_status msgemm_backward_plan_create(msgemm_handle *h, const msgemm_csr *A, const msgemm_csr *B,
                                          msgemm_backward_plan **plan) {
    if (!h || !plan) return fail(h, MSGEMM_ERR_INVALID, "NULL handle or plan");
    *plan = nullptr;
    h->nprof = 0;
    CKS(check_backward(h, A, B, nullptr, MSGEMM_PLUS_TIMES_F32));
    if (h->validate) CKS(validate_inputs(h, {A, B}));
    cudaStream_t st = h->stream;
    const long long big = std::max(A->nnz, B->nnz);
    const int wide = std::max(A->ncols, B->ncols);
    const size_t bytes = carve_size<int>((size_t)B->ncols + 1) + 2 * carve_size<int>(B->nnz) +
                         carve_size<float>(B->nnz) + carve_size<int>((size_t)A->ncols + 1) +
                         2 * carve_size<int>(A->nnz) + carve_size<float>(A->nnz) +
                         carve_size<int>((size_t)wide + 1) + carve_size<int>(big) +
                         carve_size<long long>(wide / STILE + 4) + 1024;
    msgemm_backward_plan *pl = new msgemm_backward_plan();
    pl->mem = dev_alloc(h, bytes);
    if (!pl->mem) {
        delete pl;
        return fail(h, MSGEMM_ERR_OOM, "backward plan allocation failed");
    }
    Carver cv(pl->mem);
    pl->bt_rp = cv.take<int>((size_t)B->ncols + 1);
    pl->bt_ci = cv.take<int>(B->nnz);
    pl->bt_perm = cv.take<int>(B->nnz);
    pl->bt_v = cv.take<float>(B->nnz);
    pl->at_rp = cv.take<int>((size_t)A->ncols + 1);
    pl->at_ci = cv.take<int>(A->nnz);
    pl->at_perm = cv.take<int>(A->nnz);
    pl->at_v = cv.take<float>(A->nnz);
    int *cur = cv.take<int>((size_t)wide + 1);
    int *iota = cv.take<int>(big);
    long long *tiles = cv.take<long long>(wide / STILE + 4);
    pl->device = h->device;
    pl->a_rp = A->rowptr; pl->a_ci = A->colidx; pl->am = A->nrows; pl->an = A->ncols; pl->annz = A->nnz;
    pl->b_rp = B->rowptr; pl->b_ci = B->colidx; pl->bm = B->nrows; pl->bn = B->ncols; pl->bnnz = B->nnz;
    // each transpose carries the entries' positions as its values; the
    // sorted rows then hold, per entry, where its value sits in the source
    auto build = [&](const msgemm_csr *X, int *trp, int *tci, int *tperm) -> msgemm_status {
        PScope ph(h, "plan transpose");
        CK(launch_col_counts(X->colidx, X->nnz, X->ncols, cur, st, h->nsm));
        CK(launch_excl_scan_int(cur, X->ncols, trp, tiles, st, h->nsm));
        CK(cudaMemcpyAsync(cur, trp, sizeof(int) * ((size_t)X->ncols + 1), cudaMemcpyDeviceToDevice, st));
        CK(launch_transpose_fill(X->rowptr, X->colidx, iota, 4, X->nrows, X->ncols, cur, tci, tperm, nullptr, st,
                                 h->nsm));
        CK(launch_segsort(trp, tci, tperm, 4, X->ncols, cur, st, h->nsm));
        return MSGEMM_OK;
    };
    msgemm_status rs = MSGEMM_OK;
    if (cudaSuccess != launch_iota_i32(iota, big, st, h->nsm)) rs = fail(h, MSGEMM_ERR_CUDA, "iota launch failed");
    if (rs == MSGEMM_OK) rs = build(B, pl->bt_rp, pl->bt_ci, pl->bt_perm);
    if (rs == MSGEMM_OK) rs = build(A, pl->at_rp, pl->at_ci, pl->at_perm);
    if (rs != MSGEMM_OK) {
        dev_free(h, pl->mem);
        delete pl;
        return rs;
    }
    *plan = pl;
    return MSGEMM_OK;
}

msgemm_status msgemm_backward_planned(msgemm_handle *h, msgemm_backward_plan *pl, const msgemm_csr *A,
                                      const msgemm_csr *B, const msgemm_csr *G, float *dA_vals, float *dB_vals) {
    if (!h || !pl) return fail(h, MSGEMM_ERR_INVALID, "NULL handle or plan");
    h->nprof = 0;
    CKS(check_backward(h, A, B, G, MSGEMM_PLUS_TIMES_F32));
    if (pl->device != h->device || A->rowptr != pl->a_rp || A->colidx != pl->a_ci || A->nrows != pl->am ||
        A->ncols != pl->an || A->nnz != pl->annz || B->rowptr != pl->b_rp || B->colidx != pl->b_ci ||
        B->nrows != pl->bm || B->ncols != pl->bn || B->nnz != pl->bnnz)
        return fail(h, MSGEMM_ERR_INVALID, "A or B is not the pattern the plan was made for");
    if (A->nnz > 0 && !A->values) return fail(h, MSGEMM_ERR_INVALID, "A has no values");
    if (B->nnz > 0 && !B->values) return fail(h, MSGEMM_ERR_INVALID, "B has no values");
    if (h->validate) CKS(validate_inputs(h, {A, B, G}));
    cudaStream_t st = h->stream;
    if (dA_vals) {
        {
            PScope ph(h, "gather");
            CK(launch_gather_f32(pl->bt_perm, static_cast<const float *>(B->values), B->nnz, pl->bt_v, st, h->nsm));
        }
        const msgemm_csr Bx{B->ncols, B->nrows, B->nnz, pl->bt_rp, pl->bt_ci, pl->bt_v};
        CKS(backward_dA(h, A, B, G, Bx, dA_vals));
    }
    if (dB_vals) {
        {
            PScope ph(h, "gather");
            CK(launch_gather_f32(pl->at_perm, static_cast<const float *>(A->values), A->nnz, pl->at_v, st, h->nsm));
        }
        const msgemm_csr Ax{A->ncols, A->nrows, A->nnz, pl->at_rp, pl->at_ci, pl->at_v};
        CKS(backward_dB(h, B, G, Ax, 1, dB_vals));
    }
    return MSGEMM_OK;
}

void msgemm_backward_plan_destroy(msgemm_handle *h, msgemm_backward_plan *pl) {
    if (!pl) return;
    if (h) dev_free(h, pl->mem);
    delete pl;
}

msgemm_status msgemm_run_batched(msgemm_handle *h, int nprod, const msgemm_csr *M, const int *complement,
                                 const msgemm_csr *A, const msgemm_csr *B, msgemm_semiring sr, msgemm_csr_out *C,
                                 int use_graph) {
    if (!h || nprod < 0 || (nprod > 0 && (!M || !A || !B || !C))) return fail(h, MSGEMM_ERR_INVALID, "bad arguments");
    h->nprof = 0;
    if (nprod == 0) return MSGEMM_OK;
    std::vector<ProdIn> in(nprod);
    std::vector<int> no_room(nprod);
    for (int p = 0; p < nprod; ++p) {
        CKS(check_product(h, &M[p], &A[p], &B[p], sr));
        const int comp = complement ? complement[p] != 0 : 0;
        no_room[p] = comp || h->phases == 2;
        in[p].M = &M[p]; in[p].A = &A[p]; in[p].B = &B[p]; in[p].comp = comp; in[p].C = &C[p];
    }
    h->out_allocs.clear();
    CKS(alloc_outs(h, nprod, M, no_room.data(), sr, C));
    return run_products(h, in, sr, h->validate, use_graph != 0);
}

msgemm_status msgemm_autotune(msgemm_handle *h, int nprod, const msgemm_csr *M, const int *complement,
                              const msgemm_csr *A, const msgemm_csr *B, msgemm_semiring sr, const char *cache_path) {
    if (!h || nprod < 0 || (nprod > 0 && (!M || !A || !B))) return fail(h, MSGEMM_ERR_INVALID, "bad arguments");
    for (int p = 0; p < nprod; ++p) CKS(check_product(h, &M[p], &A[p], &B[p], sr));
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, h->device));
    static const char *sr_names[3] = {"plus_times_f32", "plus_times_i64", "plus_pair_i64"};
    const std::string key = std::string(prop.name) + "|" + sr_names[sr];
    std::map<std::string, Tuned> cache;
    if (cache_path) {
        read_tuned(cache_path, cache);
        auto it = cache.find(key);
        if (it != cache.end()) {
            apply_tuned(h, it->second);
            return MSGEMM_OK;
        }
    }
    if (nprod == 0) return MSGEMM_OK;
    const int saved_profile = h->profile;
    h->profile = 0;
    Tuner tu(h, nprod, M, complement, A, B, sr);
    msgemm_status rs = tu.tune();
    h->profile = saved_profile;
    if (rs != MSGEMM_OK) return rs;
    if (cache_path) {
        cache[key] = current_tuned(h);
        if (!write_tuned(cache_path, cache)) return fail(h, MSGEMM_ERR_INVALID, "cannot write %s", cache_path);
    }
    return MSGEMM_OK;
}

msgemm_status msgemm_bc(msgemm_handle *h, const msgemm_csr *A, const int32_t *sources, int nsrc, double *centrality,
                        int32_t *levels) {
    if (!h) return MSGEMM_ERR_INVALID;
    h->nprof = 0;
    CKS(check_csr(h, A, "A", false));
    if (A->nrows != A->ncols) return fail(h, MSGEMM_ERR_SHAPE, "A is %dx%d, not square", A->nrows, A->ncols);
    if (nsrc < 0 || (nsrc > 0 && !sources) || (A->nrows > 0 && !centrality))
        return fail(h, MSGEMM_ERR_INVALID, "bad sources or output");
    cudaStream_t st = h->stream;
    const int n = A->nrows;
    if (levels) *levels = 0;
    if (n > 0) CK(cudaMemsetAsync(centrality, 0, sizeof(double) * (size_t)n, st));
    if (nsrc == 0 || n == 0) return MSGEMM_OK;
    if (h->validate) CKS(validate_inputs(h, {A}));
    {   // sources in range (host check; synchronises)
        std::vector<int32_t> hs(nsrc);
        CK(cudaMemcpyAsync(hs.data(), sources, sizeof(int32_t) * (size_t)nsrc, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int32_t x : hs)
            if (x < 0 || x >= n) return fail(h, MSGEMM_ERR_INVALID, "source %d out of range", x);
    }
    const long long nnz = A->nnz;
    const long long wpr = ((long long)n + 31) / 32;
    // every allocation of this call, released at the end (stream-ordered)
    std::vector<void *> owned;
    auto take = [&](size_t bytes) -> void * {
        void *p = dev_alloc(h, bytes);
        if (p) owned.push_back(p);
        return p;
    };
    struct Guard {
        msgemm_handle *h;
        std::vector<void *> &v;
        ~Guard() {
            for (void *p : v) dev_free(h, p);
        }
    } guard{h, owned};
    // A (forward) and A^T with rows sorted (backward right operand; its
    // transpose, A, serves pull rows) as pattern operands: every value 1
    int *at_rp = static_cast<int *>(take(sizeof(int) * ((size_t)n + 1)));
    int *at_cur = static_cast<int *>(take(sizeof(int) * ((size_t)n + 1)));
    int *at_ci = static_cast<int *>(take(sizeof(int) * (size_t)std::max(nnz, 1LL)));
    long long *tb = static_cast<long long *>(take(sizeof(long long) * ((size_t)n / STILE + 4)));
    unsigned *bm = static_cast<unsigned *>(take(sizeof(unsigned) * (size_t)(nsrc * wpr)));
    int *vrp = static_cast<int *>(take(sizeof(int) * ((size_t)nsrc + 1)));
    int *vcnt = static_cast<int *>(take(sizeof(int) * ((size_t)nsrc + 1)));
    long long *vtb = static_cast<long long *>(take(sizeof(long long) * ((size_t)nsrc / STILE + 4)));
    if (!at_rp || !at_cur || !at_ci || !tb || !bm || !vrp || !vcnt || !vtb)
        return fail(h, MSGEMM_ERR_OOM, "bc workspace allocation failed");
    CK(launch_col_counts(A->colidx, nnz, n, at_cur, st, h->nsm));
    CK(launch_excl_scan_int(at_cur, n, at_rp, tb, st, h->nsm));
    CK(cudaMemcpyAsync(at_cur, at_rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
    CK(launch_transpose_fill(A->rowptr, A->colidx, nullptr, 0, n, n, at_cur, at_ci, nullptr, nullptr, st, h->nsm));
    CK(launch_segsort(at_rp, at_ci, nullptr, 0, n, at_cur, st, h->nsm));
    CK(cudaMemsetAsync(bm, 0, sizeof(unsigned) * (size_t)(nsrc * wpr), st));
    const msgemm_csr Aone{n, n, nnz, A->rowptr, A->colidx, nullptr};
    const msgemm_csr AtOne{n, n, nnz, at_rp, at_ci, nullptr};

    // ---- forward: level 0 = the sources, level d + 1 = !visited .* (level d A)
    struct Level {
        int32_t *rp, *ci;
        long long *sigma;
        long long nnz;
    };
    std::vector<Level> lv;
    {
        Level l0;
        l0.rp = static_cast<int *>(take(sizeof(int) * ((size_t)nsrc + 1)));
        l0.ci = static_cast<int *>(take(sizeof(int) * (size_t)nsrc));
        l0.sigma = static_cast<long long *>(take(sizeof(long long) * (size_t)nsrc));
        if (!l0.rp || !l0.ci || !l0.sigma) return fail(h, MSGEMM_ERR_OOM, "bc workspace allocation failed");
        l0.nnz = nsrc;
        CK(launch_bc_sources(sources, nsrc, l0.rp, l0.ci, l0.sigma, st, h->nsm));
        lv.push_back(l0);
    }
    int *vci = nullptr;
    long long vcap = 0;
    for (;;) {
        const Level &cur = lv.back();
        // visited pattern: levels 0..d as CSR
        CK(launch_bitmap_or(cur.rp, cur.ci, nsrc, wpr, bm, st, h->nsm));
        CK(launch_bitmap_counts(bm, nsrc, wpr, vcnt, st, h->nsm));
        CK(launch_excl_scan_int(vcnt, nsrc, vrp, vtb, st, h->nsm));
        int vtot = 0;
        CK(cudaMemcpyAsync(&vtot, vrp + nsrc, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (vtot > vcap) {
            vcap = std::max<long long>(vtot, vcap * 2);
            vci = static_cast<int *>(take(sizeof(int) * (size_t)vcap));
            if (!vci) return fail(h, MSGEMM_ERR_OOM, "bc workspace allocation failed");
        }
        CK(launch_bitmap_cols(bm, nsrc, wpr, vrp, vci, st, h->nsm));
        const msgemm_csr V{nsrc, n, vtot, vrp, vci, nullptr};
        const msgemm_csr F{nsrc, n, cur.nnz, cur.rp, cur.ci, cur.sigma};
        msgemm_csr_out C;
        CKS(alloc_out(h, &V, 1, MSGEMM_PLUS_TIMES_I64, &C));
        for (void *p : {(void *)C.rowptr, (void *)C.d_nnz}) owned.push_back(p);
        std::vector<ProdIn> in(1);
        in[0].M = &V; in[0].A = &F; in[0].B = &Aone; in[0].comp = 1; in[0].C = &C;
        CKS(run_pipeline(h, in, MSGEMM_PLUS_TIMES_I64, false, false));
        for (void *p : {(void *)C.colidx, C.values}) owned.push_back(p);
        if (C.capacity == 0) break;   // no new vertex in any row (the pipeline set the exact count)
        lv.push_back(Level{C.rowptr, C.colidx, static_cast<long long *>(C.values), C.capacity});
    }
    const int D = (int)lv.size() - 1;   // deepest level
    if (levels) *levels = D + 1;

    // ---- backward: W_d = 1/sigma_d + T_d on level d, T_{d-1} = level_{d-1} .* (W_d A^T)
    // (values at each level entry's own slot), delta_{d-1} = sigma_{d-1} T_{d-1}
    float *T = nullptr;   // T_d, aligned with level d (none for the deepest level)
    for (int d = D; d >= 2; --d) {
        const Level &L = lv[d], &P = lv[d - 1];
        float *W = static_cast<float *>(take(sizeof(float) * (size_t)std::max(L.nnz, 1LL)));
        float *Tp = static_cast<float *>(take(sizeof(float) * (size_t)std::max(P.nnz, 1LL)));
        if (!W || !Tp) return fail(h, MSGEMM_ERR_OOM, "bc workspace allocation failed");
        CK(launch_bc_weight(L.sigma, T, L.nnz, W, st, h->nsm));
        CK(cudaMemsetAsync(Tp, 0, sizeof(float) * (size_t)std::max(P.nnz, 1LL), st));
        const msgemm_csr Mx{nsrc, n, P.nnz, P.rp, P.ci, nullptr};
        const msgemm_csr Wx{nsrc, n, L.nnz, L.rp, L.ci, W};
        std::vector<ProdIn> in(1);
        in[0].M = &Mx; in[0].A = &Wx; in[0].B = &AtOne; in[0].comp = 0;
        in[0].bt_rp = A->rowptr; in[0].bt_ci = A->colidx; in[0].bt_v = nullptr;
        in[0].aligned_out = Tp;
        if (P.nnz > 0) CKS(run_pipeline(h, in, MSGEMM_PLUS_TIMES_F32, false, false));
        CK(launch_bc_accum(P.ci, P.sigma, Tp, P.nnz, centrality, st, h->nsm));
        T = Tp;
    }
    // the workspace is released in stream order by the guard
    return MSGEMM_OK;
}

msgemm_status msgemm_ktruss(msgemm_handle *h, const msgemm_csr *A, int64_t k, msgemm_csr_out *T, int32_t *iterations,
                            int64_t *products) {
    if (!h || !T) return fail(h, MSGEMM_ERR_INVALID, "NULL handle or output");
    h->nprof = 0;
    CKS(check_csr(h, A, "A", false));
    if (A->nrows != A->ncols) return fail(h, MSGEMM_ERR_SHAPE, "A is %dx%d, not square", A->nrows, A->ncols);
    if (k < 0) return fail(h, MSGEMM_ERR_INVALID, "k must be >= 0");
    if (h->validate) CKS(validate_inputs(h, {A}));
    cudaStream_t st = h->stream;
    const int n = A->nrows;
    std::vector<void *> owned;
    auto take = [&](size_t bytes) -> void * {
        void *p = dev_alloc(h, bytes);
        if (p) owned.push_back(p);
        return p;
    };
    struct Guard {
        msgemm_handle *h;
        std::vector<void *> &v;
        ~Guard() {
            for (void *p : v) dev_free(h, p);
        }
    } guard{h, owned};
    int *cnt = static_cast<int *>(take(sizeof(int) * ((size_t)n + 1)));
    long long *tb = static_cast<long long *>(take(sizeof(long long) * ((size_t)n / STILE + 4)));
    long long *dsm = static_cast<long long *>(take(2 * sizeof(long long)));   // [nnz, sum]
    if (!cnt || !tb || !dsm) return fail(h, MSGEMM_ERR_OOM, "k-truss workspace allocation failed");
    struct G {
        int *rp = nullptr, *ci = nullptr;
        long long *sup = nullptr;
        long long nnz = 0;
    };
    // entries of X kept by the filter (no self loops; support >= thr when given)
    auto filter = [&](const G &X, long long thr, G &out) -> msgemm_status {
        out.rp = static_cast<int *>(take(sizeof(int) * ((size_t)n + 1)));
        if (!out.rp) return fail(h, MSGEMM_ERR_OOM, "k-truss workspace allocation failed");
        CK(launch_filter_counts(X.rp, X.ci, n, X.sup, thr, cnt, st, h->nsm));
        CK(launch_excl_scan_int(cnt, n, out.rp, tb, st, h->nsm));
        int tot = 0;
        CK(cudaMemcpyAsync(&tot, out.rp + n, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        out.nnz = tot;
        out.ci = static_cast<int *>(take(sizeof(int) * (size_t)std::max(tot, 1)));
        if (X.sup) out.sup = static_cast<long long *>(take(sizeof(long long) * (size_t)std::max(tot, 1)));
        if (!out.ci || (X.sup && !out.sup)) return fail(h, MSGEMM_ERR_OOM, "k-truss workspace allocation failed");
        CK(launch_filter_write(X.rp, X.ci, n, X.sup, thr, out.rp, out.ci, out.sup, st, h->nsm));
        return MSGEMM_OK;
    };
    G cur;
    if (n > 0) {
        G in0;
        in0.rp = const_cast<int *>(A->rowptr);
        in0.ci = const_cast<int *>(A->colidx);
        in0.nnz = A->nnz;
        CKS(filter(in0, 0, cur));   // self loops never belong to a truss
    }
    long long prod = 0;
    int it = 0;
    long long *sup = nullptr;
    while (n > 0) {
        ++it;
        // support of every edge: A .* (A A) on plus-pair, at each entry's own slot
        sup = static_cast<long long *>(take(sizeof(long long) * (size_t)std::max(cur.nnz, 1LL)));
        if (!sup) return fail(h, MSGEMM_ERR_OOM, "k-truss workspace allocation failed");
        CK(cudaMemsetAsync(sup, 0, sizeof(long long) * (size_t)std::max(cur.nnz, 1LL), st));
        if (cur.nnz > 0) {
            const msgemm_csr X{n, n, cur.nnz, cur.rp, cur.ci, nullptr};
            std::vector<ProdIn> in(1);
            in[0].M = &X; in[0].A = &X; in[0].B = &X; in[0].comp = 0;
            in[0].aligned_out = sup;
            CKS(run_pipeline(h, in, MSGEMM_PLUS_PAIR_I64, true, false));
            // products kept by the mask = the sum of the supports
            CK(cudaMemcpyAsync(dsm, &cur.nnz, sizeof(long long), cudaMemcpyHostToDevice, st));
            CK(launch_reduce_sum(MSGEMM_PLUS_PAIR_I64, sup, dsm, dsm + 1, st, h->nsm));
            long long sum = 0;
            CK(cudaMemcpyAsync(&sum, dsm + 1, sizeof(long long), cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            prod += sum;
        }
        G next;
        cur.sup = sup;
        CKS(filter(cur, k - 2, next));
        if (next.nnz == cur.nnz) break;   // nothing pruned: cur is the k-truss, sup its supports
        cur = next;
        cur.sup = nullptr;
    }
    // output: the truss's pattern with each edge's support
    memset(T, 0, sizeof *T);
    T->nrows = n;
    T->ncols = n;
    T->capacity = cur.nnz;
    T->rowptr = static_cast<int32_t *>(dev_alloc(h, sizeof(int) * ((size_t)n + 1)));
    T->colidx = static_cast<int32_t *>(dev_alloc(h, sizeof(int) * (size_t)std::max(cur.nnz, 1LL)));
    T->values = dev_alloc(h, sizeof(long long) * (size_t)std::max(cur.nnz, 1LL));
    T->d_nnz = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t)));
    if (!T->rowptr || !T->colidx || !T->values || !T->d_nnz) return fail(h, MSGEMM_ERR_OOM, "output allocation failed");
    if (n > 0) {
        CK(cudaMemcpyAsync(T->rowptr, cur.rp, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, st));
        if (cur.nnz > 0) {
            CK(cudaMemcpyAsync(T->colidx, cur.ci, sizeof(int) * (size_t)cur.nnz, cudaMemcpyDeviceToDevice, st));
            CK(cudaMemcpyAsync(T->values, sup, sizeof(long long) * (size_t)cur.nnz, cudaMemcpyDeviceToDevice, st));
        }
    } else {
        CK(cudaMemsetAsync(T->rowptr, 0, sizeof(int), st));
    }
    const long long tn = cur.nnz;
    CK(cudaMemcpyAsync(T->d_nnz, &tn, sizeof tn, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));   // host sources above; the workspace is released after this
    if (iterations) *iterations = it;
    if (products) *products = prod;
    return MSGEMM_OK;
}

msgemm_status msgemm_transpose(msgemm_handle *h, const msgemm_csr *A, int value_bytes, int sorted, msgemm_csr_out *At) {
    if (!h || !At) return MSGEMM_ERR_INVALID;
    CKS(check_csr(h, A, "A", value_bytes > 0));
    if (value_bytes != 0 && value_bytes != 4 && value_bytes != 8) return fail(h, MSGEMM_ERR_INVALID, "value_bytes");
    cudaStream_t st = h->stream;
    memset(At, 0, sizeof *At);
    At->nrows = A->ncols;
    At->ncols = A->nrows;
    At->capacity = A->nnz;
    At->rowptr = static_cast<int32_t *>(dev_alloc(h, sizeof(int) * ((size_t)A->ncols + 1)));
    At->colidx = static_cast<int32_t *>(dev_alloc(h, sizeof(int) * (size_t)std::max<long long>(A->nnz, 1)));
    At->values = value_bytes ? dev_alloc(h, (size_t)value_bytes * (size_t)std::max<long long>(A->nnz, 1)) : nullptr;
    At->d_nnz = static_cast<int64_t *>(dev_alloc(h, sizeof(int64_t)));
    if (!At->rowptr || !At->colidx || !At->d_nnz || (value_bytes && !At->values))
        return fail(h, MSGEMM_ERR_OOM, "output allocation failed");
    CKS(grow(h, h->bt, carve_size<int>((size_t)A->ncols + 1) + carve_size<long long>(A->ncols / STILE + 4)));
    Carver cb(h->bt.p);
    int *cur = cb.take<int>((size_t)A->ncols + 1);
    long long *tbuf = cb.take<long long>(A->ncols / STILE + 4);
    CK(launch_col_counts(A->colidx, A->nnz, A->ncols, cur, st, h->nsm));
    CK(launch_excl_scan_int(cur, A->ncols, At->rowptr, tbuf, st, h->nsm));
    CK(cudaMemcpyAsync(cur, At->rowptr, sizeof(int) * ((size_t)A->ncols + 1), cudaMemcpyDeviceToDevice, st));
    CK(launch_transpose_fill(A->rowptr, A->colidx, A->values, value_bytes, A->nrows, A->ncols, cur, At->colidx,
                             At->values, nullptr, st, h->nsm));
    if (sorted) CK(launch_segsort(At->rowptr, At->colidx, At->values, value_bytes, A->ncols, cur, st, h->nsm));
    int64_t nnz = A->nnz;
    CK(cudaMemcpyAsync(At->d_nnz, &nnz, sizeof nnz, cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return MSGEMM_OK;
}

msgemm_status msgemm_reduce_sum(msgemm_handle *h, const msgemm_csr_out *C, msgemm_semiring sr, void *d_sum) {
    if (!h || !C || !d_sum || !C->d_nnz) return fail(h, MSGEMM_ERR_INVALID, "bad arguments");
    PScope ph(h, "reduce");
    CK(launch_reduce_sum(sr, C->values, reinterpret_cast<const long long *>(C->d_nnz), d_sum, h->stream, h->nsm));
    return MSGEMM_OK;
}

msgemm_status msgemm_sync_status(msgemm_handle *h) {
    if (!h) return MSGEMM_ERR_INVALID;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return fail(h, MSGEMM_ERR_CUDA, "stream: %s", cudaGetErrorString(e));
    unsigned err = 0;
    CK(cudaMemcpy(&err, h->d_err, sizeof err, cudaMemcpyDeviceToHost));
    if (err) CK(cudaMemset(h->d_err, 0, sizeof err));
    if (err & ERR_TIMEOUT) return fail(h, MSGEMM_ERR_TIMEOUT, "a bounded device wait ran out");
    if (err & ERR_UNSORTED) return fail(h, MSGEMM_ERR_UNSORTED, "an input row is not strictly ascending");
    if (err & (ERR_INVALID | ERR_INTERNAL)) return fail(h, MSGEMM_ERR_INVALID, "invalid input found on the device");
    return MSGEMM_OK;
}

msgemm_status msgemm_last_error_detail(msgemm_handle *h, char *buf, size_t len) {
    if (!h || !buf || len == 0) return MSGEMM_ERR_INVALID;
    snprintf(buf, len, "%s", h->last_error.c_str());
    return MSGEMM_OK;
}

int msgemm_num_kinds(void) { return NKIND; }

msgemm_status msgemm_bin_counts(msgemm_handle *h, int64_t *counts, int n) {
    if (!h || !counts) return MSGEMM_ERR_INVALID;
    int tmp[NKIND] = {0};
    if (h->last_kind_count) {
        CK(cudaStreamSynchronize(h->stream));
        CK(cudaMemcpy(tmp, h->last_kind_count, sizeof tmp, cudaMemcpyDeviceToHost));
    }
    for (int k = 0; k < std::min(n, (int)NKIND); ++k) counts[k] = tmp[k];
    return MSGEMM_OK;
}

int msgemm_profile_count(msgemm_handle *h) { return h ? h->nprof : 0; }

msgemm_status msgemm_profile_entry(msgemm_handle *h, int idx, char *name, size_t len, float *ms) {
    if (!h || idx < 0 || idx >= h->nprof) return MSGEMM_ERR_INVALID;
    if (name && len) snprintf(name, len, "%s", h->prof[idx].name.c_str());
    if (ms) {
        CK(cudaEventSynchronize(h->prof[idx].b));
        CK(cudaEventElapsedTime(ms, h->prof[idx].a, h->prof[idx].b));
    }
    return MSGEMM_OK;
}

msgemm_status msgemm_last_row_kinds(msgemm_handle *h, uint8_t *kinds, int64_t nrows) {
    if (!h || (!kinds && nrows > 0)) return MSGEMM_ERR_INVALID;
    if (nrows != h->last_R) return fail(h, MSGEMM_ERR_INVALID, "last call had %lld rows", h->last_R);
    if (nrows == 0) return MSGEMM_OK;
    CK(cudaStreamSynchronize(h->stream));
    CK(cudaMemcpy(kinds, h->last_kind, (size_t)nrows, cudaMemcpyDeviceToHost));
    return MSGEMM_OK;
}

int64_t msgemm_kernel_launches(void) { return g_kernel_launches.load(); }

void msgemm_destroy(msgemm_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    for (auto &ph : h->prof) {
        cudaEventDestroy(ph.a);
        cudaEventDestroy(ph.b);
    }
    if (h->gexec) cudaGraphExecDestroy(h->gexec);
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    for (Buf *b : {&h->rows, &h->small, &h->tmp, &h->bt, &h->cur, &h->prods, &h->tix, &h->gbuf, &h->thi, &h->gpbuf})
        dev_free(h, b->p);
    delete h;
}

}  // extern "C"
