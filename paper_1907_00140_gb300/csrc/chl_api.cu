// C ABI of libchl.so (declared in include/chl.h): argument checks, device
// memory, the build driver (graph preparation, persistent tree launch with
// retry on a full label buffer, label assembly) and the query entry point.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "chl_common.cuh"


namespace chl {

static thread_local char g_err[512] = "";

chl_status set_error(chl_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

chl_status cuda_status(cudaError_t e, const char *what) {
    // the failed call also left e in the thread's last-error state (an
    // allocation failure is not sticky): consume it, or the next launch check
    // of a later call would report it again
    (void)cudaGetLastError();
    return set_error(e == cudaErrorMemoryAllocation ? CHL_ENOMEM : CHL_ECUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

cudaError_t exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, cudaStream_t s,
                               int *launches);

// Device memory of the library's stream-ordered allocations comes from one
// pool per device that keeps up to POOL_KEEP bytes cached after a
// synchronisation (the default pool keeps none, so each build would map its
// gigabytes of tree-slot state again).
constexpr uint64_t POOL_KEEP = uint64_t(32) << 30;

cudaError_t dmalloc(void **ptr, size_t bytes, cudaStream_t s) {
    constexpr int MAXDEV = 64;
    static std::mutex mu;
    static cudaMemPool_t pools[MAXDEV] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e) return e;
    if (dev < 0 || dev >= MAXDEV) return cudaMallocAsync(ptr, bytes, s);
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lk(mu);
        if (!pools[dev]) {
            cudaMemPoolProps props{};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            cudaMemPool_t p = nullptr;
            e = cudaMemPoolCreate(&p, &props);
            if (e) return e;
            uint64_t keep = POOL_KEEP;
            e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
            if (e) {
                cudaMemPoolDestroy(p);
                return e;
            }
            pools[dev] = p;
        }
        pool = pools[dev];
    }
    return cudaMallocFromPoolAsync(ptr, bytes, pool, s);
}

int device_sms() {
    constexpr int MAXDEV = 64;
    static std::atomic<int> cached[MAXDEV];
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < MAXDEV && (v = cached[dev].load(std::memory_order_relaxed)) > 0) return v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) return 1;
    if (dev >= 0 && dev < MAXDEV) cached[dev].store(v, std::memory_order_relaxed);
    return v;
}

namespace {

// device control block of one tree launch; the two counters every tree
// updates sit on cache lines of their own
struct Control {
    alignas(128) unsigned int next_root;
    alignas(128) unsigned long long out_count;
    unsigned long long out_valid;
    alignas(128) unsigned int failed_count;
    unsigned int list_n;  // roots listed by the trivial-root split
    int flags[2];
    unsigned long long stats[7];
};

void bind_control(TreeLaunch &tl, Control *ctl) {
    tl.out_count = &ctl->out_count;
    tl.out_valid = &ctl->out_valid;
    tl.next_root = &ctl->next_root;
    tl.failed_count = &ctl->failed_count;
    tl.flags = ctl->flags;
    tl.stats = ctl->stats;
}

// records of an attempt that are whole trees
uint64_t records_kept(const Control &c) { return c.flags[1] ? c.out_valid : c.out_count; }

// label record buffers (vertex, hub, distance, optional parent): moved to a
// capacity of ncap records, keeping the first T
cudaError_t grow_records(void **bufs, int nbufs, uint64_t T, uint64_t ncap, cudaStream_t s) {
    for (int k = 0; k < nbufs; ++k) {
        void *nb = nullptr;
        cudaError_t e = dmalloc(&nb, ncap * 4, s);
        if (!e && T) e = cudaMemcpyAsync(nb, bufs[k], T * 4, cudaMemcpyDeviceToDevice, s);
        if (e) {
            if (nb) cudaFreeAsync(nb, s);
            return e;
        }
        cudaFreeAsync(bufs[k], s);
        bufs[k] = nb;
    }
    return cudaSuccess;
}

// expansion rounds one tree may take (far above any real tree)
constexpr uint32_t DEFAULT_ROUND_LIMIT = 1u << 26;
// a label-pruned phase whose trees averaged fewer expansions than this hands
// the later phases to the small-tree launch
constexpr uint32_t DEFAULT_SMALL_TREE_EXPANSIONS = 8192;
// a label-pruned phase after one whose trees averaged at least this share of
// the vertices takes the narrow big-tree bucket width (measured on R-MAT
// scale 18 and 21: the phases after trees of 0.48 n and more gained, those
// after trees of 0.43 n and less lost)
constexpr double BIG_TREE_COVER = 0.45;
// shared memory per tree slot for the root's table distances by hub position in
// the label-pruned phases: phases whose table holds at most 16,384 hubs look
// each entry up with one load instead of a hash probe
constexpr uint32_t ROOT_ARRAY_BYTES = 64u << 10;

struct Params {
    int tpt;
    int tpt_lt;          // threads per tree in the label-pruned phases
    int slots_lt;        // ... and their slots
    uint32_t fin_words_lt;
    uint32_t aux_lt;     // auxiliary shared memory of those phases (staging or root distances)
    // label-pruned phases of small trees (after a phase whose trees averaged
    // fewer than small_exp expansions): smaller blocks, more trees per SM
    int tpt_sm, slots_sm;
    uint32_t fin_words_sm, aux_sm, small_exp;
    uint32_t nwin_sm;  // window buckets of the small-tree launch (its trees span few buckets)
    uint32_t stage_want; // staging of the queried lists, as requested (0 = none)
    uint32_t round_limit;
    uint32_t delta;
    uint32_t delta_lt;  // bucket width of the phases that prune with the label table
    uint32_t delta_big; // ... of such a phase after big trees (0: no separate width)
    uint32_t nwin;
    int slots;
    int kb;  // bytes per tree key: 4 or 8
    uint32_t eta;  // Common Label Table hubs (0 = no table)
    uint32_t fin_words;  // settled-filter bitmap words per CTA
    uint32_t w_min;
    uint32_t n;
    int max_slots() const { return std::max(slots, std::max(slots_lt, slots_sm)); }
    // list words per vertex over all slots, the largest of the launches' layouts
    size_t list_words() const {
        return std::max(size_t(std::max(slots, slots_lt)) * (4 + nwin), size_t(slots_sm) * (4 + nwin_sm));
    }
};

// Untuned defaults of the search parameters from graph statistics (chl_tune
// measures instead). Bucket width: low-diameter graphs with many vertices per
// unit of distance (mean degree >= 8, the scale-free families) need narrow
// buckets, since early termination is decided at bucket granularity; sparse
// high-diameter graphs (road-like) want wide buckets, so that a tree needs few
// bucket rounds.
Params choose_params(const RankGraph &g, const chl_build_opts &o, int sms, size_t free_bytes) {
    Params p;
    p.tpt = o.threads_per_tree ? o.threads_per_tree : 1024;
    const double mean_deg = g.n ? double(g.m2) / double(g.n) : 0.0;
    const double dflt = mean_deg >= 8.0 ? g.w_mean / 128.0 : 2.0 * g.w_mean;
    uint32_t d = 1;  // default: the power of two nearest to dflt
    while (double(d) * 1.5 < dflt && d < (1u << 30)) d <<= 1;
    if (o.bucket_delta > 0) d = uint32_t(o.bucket_delta);
    p.delta = d;
    uint32_t dl = 1;
    while (double(dl) * 1.5 < 2.0 * g.w_mean && dl < (1u << 30)) dl <<= 1;
    p.delta_lt = o.pruned_bucket_delta > 0 ? uint32_t(o.pruned_bucket_delta) : dl;
    p.delta_big = o.big_tree_bucket_delta > 0   ? uint32_t(o.big_tree_bucket_delta)
                  : o.big_tree_bucket_delta < 0 ? 0u
                                                : std::max<uint32_t>(1u, p.delta_lt / 16);
    p.nwin = o.window_buckets > 0 ? uint32_t(o.window_buckets) : 32;
    // 4-byte keys hold distances up to 2^31 - 2; every tentative distance of a
    // tree search is at most w_max * n (a simple path plus one arc)
    const bool narrow_fits = double(g.w_max) * double(g.n) <= double(0x7FFFFFFE);
    // parents ride in the low 31 bits of an 8-byte key
    p.kb = (narrow_fits && !(o.flags & (CHL_FLAG_WIDE_KEYS | CHL_FLAG_PARENTS))) ? 4 : 8;
    {
        uint32_t st0 = 0;
        plant_smem_split(p.tpt, g.n, 0, &p.fin_words, &st0);
    }
    {
        const int want = o.common_hubs == 0 ? 16 : o.common_hubs;  // the paper's eta = 16
        p.eta = want < 0 ? 0u : (uint32_t(want) < g.n ? uint32_t(want) : g.n);
    }
    p.w_min = g.w_min ? g.w_min : 1;
    p.n = g.n;
    p.tpt_lt = o.pruned_threads_per_tree ? o.pruned_threads_per_tree : p.tpt;
    // the label-pruned phases' auxiliary area: the staging of queried lists
    // when asked for, else the root's table distances by hub position
    p.stage_want = o.query_stage_kb > 0 ? uint32_t(o.query_stage_kb) << 10 : 0u;
    plant_smem_split(p.tpt_lt, g.n, p.stage_want ? p.stage_want : ROOT_ARRAY_BYTES, &p.fin_words_lt,
                     &p.aux_lt);
    p.round_limit = o.round_limit ? o.round_limit : DEFAULT_ROUND_LIMIT;
    int per_sm = plant_max_slots_per_sm(p.tpt, p.fin_words, 0);
    if (per_sm < 1) per_sm = 1;
    int per_sm_lt = plant_max_slots_per_sm(p.tpt_lt, p.fin_words_lt, p.aux_lt);
    p.tpt_sm = o.small_threads_per_tree ? o.small_threads_per_tree : std::min(p.tpt_lt, 256);
    p.nwin_sm = std::min<uint32_t>(p.nwin, 8);
    p.small_exp = o.small_tree_expansions ? o.small_tree_expansions : DEFAULT_SMALL_TREE_EXPANSIONS;
    plant_smem_split(p.tpt_sm, g.n, p.stage_want ? p.stage_want : ROOT_ARRAY_BYTES, &p.fin_words_sm,
                     &p.aux_sm);
    int per_sm_sm = plant_max_slots_per_sm(p.tpt_sm, p.fin_words_sm, p.aux_sm);
    if (per_sm_sm < 1) per_sm_sm = 1;
    long long slots_sm = o.slots > 0 ? o.slots : (long long)sms * per_sm_sm;
    if (per_sm_lt < 1) per_sm_lt = 1;
    long long slots = o.slots > 0 ? o.slots : (long long)sms * per_sm;
    long long slots_lt = o.slots > 0 ? o.slots : (long long)sms * per_sm_lt;
    // slot state per vertex: key + round tag 4 + (4 + nwin) lists of 4 bytes,
    // + 4 for the root's labels of a hybrid build
    const double per_slot = (p.kb + 8.0 + 4.0 * (4 + p.nwin)) * double(g.n) + 64.0;
    const double budget = 0.35 * double(free_bytes);
    long long cap = (long long)(budget / per_slot);
    if (o.slots <= 0 && slots > cap) slots = cap;
    if (slots < 1) slots = 1;
    if (o.slots <= 0 && slots_lt > cap) slots_lt = cap;
    if (slots_lt < 1) slots_lt = 1;
    {
        const double per_slot_sm = (p.kb + 8.0 + 4.0 * (4 + p.nwin_sm)) * double(g.n) + 64.0;
        const long long cap_sm = (long long)(budget / per_slot_sm);
        if (o.slots <= 0 && slots_sm > cap_sm) slots_sm = cap_sm;
    }
    if (slots_sm < 1) slots_sm = 1;
    p.slots_sm = int(slots_sm);
    p.slots = int(slots);
    p.slots_lt = int(slots_lt);
    return p;
}

struct DevBuf {
    void *p = nullptr;
    cudaStream_t s = nullptr;
    ~DevBuf() {
        if (p) cudaFreeAsync(p, s);
    }
    void release() {
        if (p) cudaFreeAsync(p, s);
        p = nullptr;
    }
};

void set_delta(TreeLaunch &tl, uint32_t delta) {
    tl.delta = delta;
    tl.delta_shift = -1;
    for (int b = 0; b < 32; ++b)
        if (delta == (1u << b)) tl.delta_shift = b;
}

// Per-slot search state of the tree kernel, in its idle form: keys all ones
// (unreached), tags and instance counters 0.
struct SlotState {
    DevBuf key, tags, lists, ctr;
    cudaError_t alloc(const Params &P, uint32_t n, cudaStream_t s) {
        key.s = tags.s = lists.s = ctr.s = s;
        const size_t sn = size_t(P.max_slots()) * n;
        cudaError_t e;
        if ((e = dmalloc(&key.p, sn * P.kb, s))) return e;
        if ((e = cudaMemsetAsync(key.p, 0xFF, sn * P.kb, s))) return e;
        if ((e = dmalloc(&tags.p, sn * 4, s))) return e;
        if ((e = cudaMemsetAsync(tags.p, 0, sn * 4, s))) return e;
        if ((e = dmalloc(&lists.p, P.list_words() * n * 4, s))) return e;
        if ((e = dmalloc(&ctr.p, size_t(P.max_slots()) * 16, s))) return e;
        if ((e = cudaMemsetAsync(ctr.p, 0, size_t(P.max_slots()) * 16, s))) return e;
        return cudaSuccess;
    }
    void fill(const Params &P, uint32_t n, TreeLaunch &tl) const {
        set_delta(tl, P.delta);
        tl.nwin = P.nwin;
        tl.round_limit = P.round_limit;
        tl.key = key.p;
        tl.key_bytes = P.kb;
        tl.w_min = P.w_min;
        tl.fin_words = P.fin_words;
        tl.fin_bits = P.fin_words * 32 < n ? P.fin_words * 32 : n;
        tl.rtag = (uint32_t *)tags.p;
        tl.lists = (uint32_t *)lists.p;
        tl.slot_ctr = (uint32_t *)ctr.p;
        tl.dyn_slots = 1;  // each CTA takes a free slot, so that launches may overlap
    }
    void release() {
        key.release();
        tags.release();
        lists.release();
        ctr.release();
    }
};

// The next phase's first trees, started in the tail of a label-pruned phase on
// a second stream: while the phase's last trees run, most SMs would idle. They
// prune with the current phase's table (its hubs are a rank-closed set, so
// the labels are the same; the next phase's fresher table would only prune
// more), take roots from the counter the rest of their phase then shares, and
// write their labels to buffers of their own, appended after their phase, so
// that every phase's records stay one range for the table's growth. They stop
// claiming roots once the current phase's launch is done.
struct Filler {
    DevBuf ctl, fail, roots, ov, oh, od, op, stop;
    uint64_t cap = 0;     // records the output buffers hold
    uint32_t roots_cap = 0;
    bool active = false;
    uint32_t pb = 0, pe = 0;  // the phase whose first trees these are
    cudaEvent_t ev_clear = nullptr, ev_split = nullptr, ev_done = nullptr;
    LabelTable old;           // a table grown while these trees read it: freed after them
    Control hc{};
};

// default expansions per label of a phase above which the next phases prune
// with the label table of the earlier ones
constexpr double PSI_TH = 16.0;
// ... or the share of a phase's expansions that the Common Label Table pruned
// above which they do: where the top 16 hubs already cut that much, the labels
// of every earlier hub cut far more and the per-vertex query pays
constexpr double CLT_PRUNE_TH = 0.10;
// ... or, right after the first phase (one tree per slot), the labels it
// produced per arc of the graph stay below this: scale-free graphs, whose top
// hubs cover most shortest paths, give 1.4 to 3 and gain from pruning with
// those labels at once; grids give above 10 and lose by it
constexpr double SWITCH_RATIO = 6.0;

// Common Label Table (Sec. 5.3): all labels of the `hubs` most important
// vertices, as a dense [n][stride] table of distances (all ones = no label).
struct CommonTable {
    DevBuf buf;
    uint32_t hubs = 0, stride = 0;
    void fill(TreeLaunch &tl) const {
        tl.hc = (const uint32_t *)buf.p;
        tl.hc_hubs = buf.p ? hubs : 0;
        tl.hc_stride = stride;
    }
};

}  // namespace
}  // namespace chl

using namespace chl;

#define CUDA_TRY(x)                                                              \
    do {                                                                         \
        cudaError_t e__ = (x);                                                   \
        if (e__ != cudaSuccess) {                                                \
            st = cuda_status(e__, #x);                                           \
            goto done;                                                           \
        }                                                                        \
    } while (0)

// entry of a call that launches work: the calling thread's CUDA last-error
// state is cleared, so that an error left by earlier, unrelated work is not
// reported as a failed launch of this call
#define ENTER()                 \
    do {                        \
        g_err[0] = 0;           \
        (void)cudaGetLastError(); \
    } while (0)

namespace {

// Build the Common Label Table: the trees of roots [0, P.eta), unpruned, into
// a scratch label buffer (at most n labels per tree, so it always fits), then
// one scatter of their records into the table.
chl_status build_common_table(const RankGraph &rg, const Params &P, const SlotState &slot,
                              cudaStream_t s, CommonTable &t, int *launches,
                              unsigned long long *agg) {
    chl_status st = CHL_OK;
    const uint32_t n = rg.n;
    DevBuf b_ov, b_oh, b_od, b_ctl, b_fail;
    b_ov.s = b_oh.s = b_od.s = b_ctl.s = b_fail.s = t.buf.s = s;
    const uint64_t cap = uint64_t(P.eta) * n + 1;
    Control hc{};
    Control *ctl = nullptr;
    TreeLaunch tl{};
    t.hubs = P.eta;
    t.stride = (P.eta + 3) & ~3u;
    CUDA_TRY(dmalloc(&t.buf.p, size_t(n) * t.stride * 4, s));
    CUDA_TRY(cudaMemsetAsync(t.buf.p, 0xFF, size_t(n) * t.stride * 4, s));
    CUDA_TRY(dmalloc(&b_ov.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_oh.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_od.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_fail.p, (size_t(P.eta) + 1) * 4, s));
    CUDA_TRY(dmalloc(&b_ctl.p, sizeof(Control), s));
    CUDA_TRY(cudaMemsetAsync(b_ctl.p, 0, sizeof(Control), s));
    ctl = (Control *)b_ctl.p;
    tl.n = n;
    tl.row = rg.row;
    tl.arc = rg.arc;
    tl.vert_at = rg.vert_at;
    tl.root_list = nullptr;
    tl.root_begin = 0;
    tl.root_count = P.eta;
    slot.fill(P, n, tl);  // no table: these trees are not pruned
    tl.out_v = (uint32_t *)b_ov.p;
    tl.out_h = (uint32_t *)b_oh.p;
    tl.out_d = (uint32_t *)b_od.p;
    tl.out_cap = cap;
    bind_control(tl, ctl);
    tl.failed = (uint32_t *)b_fail.p;
    CUDA_TRY(launch_plant_trees(tl, P.tpt, P.slots, s));
    ++*launches;
    CUDA_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hc.flags[0] == ERR_DIST_OVERFLOW) {
        st = set_error(CHL_EOVERFLOW, "a shortest distance reaches UINT32_MAX");
        goto done;
    }
    if (hc.flags[0] || hc.flags[1]) {
        st = set_error(CHL_ETIMEOUT, "common label table trees failed (code %d)", hc.flags[0]);
        goto done;
    }
    if (agg)
        for (int k = 0; k < 7; ++k) agg[k] += hc.stats[k];
    CUDA_TRY(launch_clt_fill((const uint32_t *)b_ov.p, (const uint32_t *)b_oh.p,
                             (const uint32_t *)b_od.p, hc.out_count, rg.pos_of, (uint32_t *)t.buf.p,
                             t.stride, t.hubs, s));
    ++*launches;
done:
    return st;
}

// the same table from the records of a build whose first trees were the
// table's roots (every label of hubs below eta is among the count records)
chl_status table_from_records(const RankGraph &rg, const Params &P, const uint32_t *ov,
                              const uint32_t *oh, const uint32_t *od, uint64_t count,
                              cudaStream_t s, CommonTable &t, int *launches) {
    chl_status st = CHL_OK;
    const uint32_t n = rg.n;
    t.buf.s = s;
    t.hubs = P.eta;
    t.stride = (P.eta + 3) & ~3u;
    CUDA_TRY(dmalloc(&t.buf.p, size_t(n) * t.stride * 4, s));
    CUDA_TRY(cudaMemsetAsync(t.buf.p, 0xFF, size_t(n) * t.stride * 4, s));
    CUDA_TRY(launch_clt_fill(ov, oh, od, count, rg.pos_of, (uint32_t *)t.buf.p, t.stride, t.hubs, s));
    ++*launches;
done:
    return st;
}

}  // namespace

// the labels live on the current device; another device's pointers would be
// read by the kernels of this call
static chl_status check_device(const chl_labels *L) {
    int dev = -1;
    const cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
    if (dev != L->device)
        return set_error(CHL_EINVAL, "labels live on device %d, the current device is %d", L->device, dev);
    return CHL_OK;
}

#define CHECK_DEVICE(L)                          \
    do {                                         \
        const chl_status d__ = check_device(L);  \
        if (d__ != CHL_OK) return d__;           \
    } while (0)

extern "C" const char *chl_last_error(void) { return g_err; }

extern "C" const char *chl_version(void) { return "chl-gb300 0.2 (sm_103a)"; }

extern "C" chl_status chl_build(const chl_csr *g, const uint32_t *rank, const chl_build_opts *opts,
                                void *stream, chl_labels **out) {
    ENTER();
    if (!out) return set_error(CHL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!g || !rank) return set_error(CHL_EINVAL, "graph or rank is NULL");
    if (g->n == 0) return set_error(CHL_EINVAL, "graph has no vertices");
    if (g->n >= 0x7FFFFFFFu) return set_error(CHL_EINVAL, "n must be < 2^31");
    if (!g->row_ptr || (g->num_arcs && (!g->col || !g->w)))
        return set_error(CHL_EINVAL, "graph arrays are NULL");
    if (g->mem != CHL_MEM_DEVICE && g->mem != CHL_MEM_HOST)
        return set_error(CHL_EINVAL, "unknown memory kind");
    chl_build_opts o{};
    if (opts) o = *opts;
    const uint32_t n = g->n;
    const uint32_t rb = o.root_begin, re = o.root_end ? o.root_end : n;
    if (rb > re || re > n) return set_error(CHL_EINVAL, "root range [%u,%u) outside [0,%u)", rb, re, n);
    if (o.threads_per_tree && (o.threads_per_tree < 32 || o.threads_per_tree > 1024 ||
                               (o.threads_per_tree & (o.threads_per_tree - 1))))
        return set_error(CHL_EINVAL, "threads_per_tree must be a power of two in [32, 1024]");
    if (o.small_threads_per_tree && (o.small_threads_per_tree < 32 || o.small_threads_per_tree > 1024 ||
                                     (o.small_threads_per_tree & (o.small_threads_per_tree - 1))))
        return set_error(CHL_EINVAL, "small_threads_per_tree must be a power of two in [32, 1024]");
    if (o.pruned_threads_per_tree &&
        (o.pruned_threads_per_tree < 32 || o.pruned_threads_per_tree > 1024 ||
         (o.pruned_threads_per_tree & (o.pruned_threads_per_tree - 1))))
        return set_error(CHL_EINVAL, "pruned_threads_per_tree must be a power of two in [32, 1024]");
    if (o.window_buckets && (o.window_buckets < 2 || o.window_buckets > 64))
        return set_error(CHL_EINVAL, "window_buckets must be in [2,64]");
    if (o.mode != 0 && o.mode != 1) return set_error(CHL_EINVAL, "mode must be 0 or 1");
    if (o.common_hubs > int32_t(CHL_MAX_COMMON_HUBS))
        return set_error(CHL_EINVAL, "common_hubs must be at most %d", CHL_MAX_COMMON_HUBS);
    if (o.bucket_delta < 0 || o.slots < 0 || o.pruned_bucket_delta < 0 || !(o.psi_threshold >= 0.0f) ||
        o.switch_ratio != o.switch_ratio || o.query_stage_kb < 0 || o.query_stage_kb > 4096)
        return set_error(CHL_EINVAL, "negative or out-of-range option");
    if (o.flags & ~int32_t(CHL_FLAG_WIDE_KEYS | CHL_FLAG_PARENTS | CHL_FLAG_NO_HYBRID |
                           CHL_FLAG_DENSE_ROOT_LABELS))
        return set_error(CHL_EINVAL, "unknown bit in flags");

    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    int launches = 0;
    int dev = 0, sms = 0;
    size_t free_b = 0, total_b = 0;
    const uint64_t m2 = g->num_arcs;
    const uint64_t *d_row = g->row_ptr;
    const uint32_t *d_col = g->col, *d_w = g->w, *d_rank = rank;
    DevBuf b_row, b_col, b_w, b_rank, b_ctl, b_ov, b_oh, b_od, b_op, b_fail, b_roots, b_ltroot;
    const bool parents = (o.flags & CHL_FLAG_PARENTS) != 0;
    uint32_t *csr_parent = nullptr;
    SlotState slot;
    CommonTable table;
    RankGraph rg;
    Params P{};
    Control hc{};
    Control *ctl = nullptr;
    LabelCSR csr;
    uint64_t cap = 0;
    uint64_t T = 0;
    int too_long = 0;
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    float ms_total = 0, ms_tree = 0, ms_sort = 0, ms_table = 0;
    bool with_table = false;
    chl_labels *L = nullptr;
    unsigned long long agg[7] = {0, 0, 0, 0, 0, 0, 0};
    std::vector<uint32_t> pending;  // roots still to build (after a full buffer)
    std::vector<std::pair<uint32_t, uint32_t>> phases;
    LabelTable lt;  // labels of earlier phases (hybrid)
    bool use_lt = false, hybrid = false, hybrid_off = false;
    bool small = false;  // later label-pruned phases run the small-tree launch
    bool big = false;    // the previous phase's trees were big (BIG_TREE_COVER)
    uint64_t lt_phases = 0, small_phases = 0, overlapped = 0;
    uint64_t lt_records = 0;  // output records the label table holds
    const double psi_th = o.psi_threshold > 0.0f ? double(o.psi_threshold) : PSI_TH;
    uint32_t claimed_upto = 0;
    bool first = true;
    Filler fill[2];                  // next-phase trees in a phase's tail, by phase parity
    cudaStream_t s2 = nullptr;       // ... and their stream
    bool overlap = false;
    bool listed = false;             // the current attempt runs from the device root list
    std::vector<uint32_t> list_h;    // ... whose host copy, when needed
    uint32_t list_n = 0;
    // CHL_TRACE=1 prints one line per phase to stderr (host clock around the
    // stream synchronisations the build already makes)
    const bool trace = std::getenv("CHL_TRACE") && std::getenv("CHL_TRACE")[0] == '1';
    auto now_ms = [] {
        return std::chrono::duration<double, std::milli>(
                   std::chrono::steady_clock::now().time_since_epoch()).count();
    };
    double t_ph = 0;

    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    for (auto &e : ev) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventRecord(ev[0], s));
    b_row.s = b_col.s = b_w.s = b_rank.s = b_ctl.s = s;
    b_ov.s = b_oh.s = b_od.s = b_op.s = b_fail.s = b_roots.s = b_ltroot.s = s;

    // inputs on the device
    if (g->mem == CHL_MEM_HOST) {
        CUDA_TRY(dmalloc(&b_row.p, (size_t(n) + 1) * 8, s));
        CUDA_TRY(dmalloc(&b_col.p, (m2 ? m2 : 1) * 4, s));
        CUDA_TRY(dmalloc(&b_w.p, (m2 ? m2 : 1) * 4, s));
        CUDA_TRY(dmalloc(&b_rank.p, size_t(n) * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_row.p, g->row_ptr, (size_t(n) + 1) * 8, cudaMemcpyHostToDevice, s));
        if (m2) {
            CUDA_TRY(cudaMemcpyAsync(b_col.p, g->col, m2 * 4, cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(b_w.p, g->w, m2 * 4, cudaMemcpyHostToDevice, s));
        }
        CUDA_TRY(cudaMemcpyAsync(b_rank.p, rank, size_t(n) * 4, cudaMemcpyHostToDevice, s));
        d_row = (const uint64_t *)b_row.p;
        d_col = (const uint32_t *)b_col.p;
        d_w = (const uint32_t *)b_w.p;
        d_rank = (const uint32_t *)b_rank.p;
    }
    {
        uint64_t last = 0;
        CUDA_TRY(cudaMemcpyAsync(&last, d_row + n, 8, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        if (last != m2) {
            st = set_error(CHL_EINVAL, "row_ptr[n] = %llu differs from num_arcs = %llu",
                           (unsigned long long)last, (unsigned long long)m2);
            goto done;
        }
    }
    st = prepare_graph(n, m2, d_row, d_col, d_w, d_rank, rg, s, &launches);
    if (st != CHL_OK) goto done;

    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    {
        chl_build_opts oq = o;
        if (o.mode == 1 && !oq.threads_per_tree) oq.threads_per_tree = 512;  // plain form: one CTA
        P = choose_params(rg, oq, sms, free_b);
        if (o.mode == 1) {
            P.slots = 1;
            P.slots_lt = 1;
            P.tpt_lt = P.tpt;
            plant_smem_split(P.tpt_lt, rg.n, P.stage_want ? P.stage_want : ROOT_ARRAY_BYTES,
                             &P.fin_words_lt, &P.aux_lt);
            P.slots_sm = 1;
            P.tpt_sm = P.tpt;
            P.nwin_sm = P.nwin;
            P.fin_words_sm = P.fin_words_lt;
            P.aux_sm = P.aux_lt;
        }
    }

    CUDA_TRY(slot.alloc(P, n, s));
    CUDA_TRY(dmalloc(&b_ctl.p, sizeof(Control), s));
    ctl = (Control *)b_ctl.p;
    CUDA_TRY(dmalloc(&b_fail.p, size_t(re - rb + 1) * 4, s));
    CUDA_TRY(dmalloc(&b_roots.p, size_t(re - rb + 1) * 4, s));

    // label buffer: an estimate, grown (x2) when a tree does not fit
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    // label buffer: up to 512 labels per vertex of the graph (within a quarter
    // of the free memory), above the average list length of the workloads
    // measured (104 to 460); it doubles and the roots that did not fit are
    // rebuilt
    cap = o.label_capacity;
    if (!cap) {
        // a tree labels at most n vertices, and the whole labeling averages
        // fewer than 512 labels per vertex on the workloads measured
        cap = std::min(uint64_t(re - rb) * n, uint64_t(n) * 512) + 1024;
        const uint64_t fit = uint64_t(0.25 * double(free_b)) / 12;
        if (cap > fit) cap = fit;
        if (cap < 1024) cap = 1024;
    }
    if (cap < 1) cap = 1;
    CUDA_TRY(dmalloc(&b_ov.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_oh.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_od.p, cap * 4, s));
    if (parents) CUDA_TRY(dmalloc(&b_op.p, cap * 4, s));

    CUDA_TRY(cudaEventRecord(ev[1], s));
    // Hybrid phases (Sec. 5.2): a build that starts at the top root runs its
    // roots in phases; the trees of a phase also prune with every label of all
    // earlier phases (a rank-closed hub set, so the labels stay canonical)
    // once the switch has fired. Other builds run as one phase.
    hybrid = rb == 0 && P.eta && !(o.flags & CHL_FLAG_NO_HYBRID) && re > P.eta;
    overlap = hybrid && o.mode == 0 && o.overlap_phases >= 0;
    // the Common Label Table is needed when some requested tree lies outside
    // it; a hybrid build takes it from its first phase instead
    if (P.eta && re > P.eta && !hybrid) {
        st = build_common_table(rg, P, slot, s, table, &launches, nullptr);
        if (st != CHL_OK) goto done;
        with_table = true;
    }
    CUDA_TRY(cudaEventRecord(ev[4], s));
    phases.clear();
    // a hybrid build's first phase is one tree per slot (at least the table's
    // roots), built without any table
    phases.push_back(hybrid ? std::make_pair(0u, uint32_t(std::min<uint64_t>(
                                                     re, std::max<uint64_t>(P.eta, uint64_t(P.slots)))))
                            : std::make_pair(rb, re));
    for (size_t ph = 0; ph < phases.size(); ++ph) {
    const uint32_t pb = phases[ph].first, pe = phases[ph].second;
    const uint64_t exp0 = agg[0], T0 = T, arc0 = agg[1], pr0 = agg[6], rd0 = agg[4], bk0 = agg[5];
    const uint64_t tr0 = agg[3], triv0 = agg[2];
    const bool ph_small = small;
    const bool ph_narrow = big && P.delta_big && lt.offsets;
    const int ph_lt = lt.offsets ? 1 : 0;
    if (trace) t_ph = now_ms();
    if (lt.offsets) ++lt_phases;
    if (small) ++small_phases;
    first = true;
    pending.clear();
    // a filler launched in the previous phase's tail built this phase's first trees
    Filler &fin = fill[(ph + 1) & 1];
    const bool from_filler = fin.active && fin.pb == pb && fin.pe == pe;
    bool filler_merged = false;
    for (Filler &f : fill) {
        if (f.active && !(from_filler && &f == &fin)) {
            // trees for a phase that did not follow: their roots are built
            // again by their own phase, their labels are dropped
            CUDA_TRY(cudaEventSynchronize(f.ev_done));
            f.active = false;
            free_table(f.old, s);
        }
    }
    for (int attempt = 0;; ++attempt) {
        TreeLaunch tl{};
        tl.n = n;
        tl.row = rg.row;
        tl.arc = rg.arc;
        tl.vert_at = rg.vert_at;
        slot.fill(P, n, tl);
        table.fill(tl);
        if (lt.offsets) {
            tl.lt_off = lt.offsets;
            tl.lt_e = lt.e;
            tl.lt_hubs = pb;
            tl.lt_root = (uint32_t *)b_ltroot.p;
            tl.lt_hash_max = (o.flags & CHL_FLAG_DENSE_ROOT_LABELS) ? 0 : 0xFFFFFFFFu;
            set_delta(tl, big && P.delta_big ? P.delta_big : P.delta_lt);
            // dynamic shared memory of this phase's launch: the root's table
            // distances need 4 bytes per hub of the table (or the staging
            // area when asked for); the settled bitmap takes the rest
            {
                const int tpt = small ? P.tpt_sm : P.tpt_lt;
                const uint32_t need = ((pb * 4u) + 127u) & ~127u;
                uint32_t want = P.stage_want ? P.stage_want : (need <= ROOT_ARRAY_BYTES ? need : 0u);
                plant_smem_split(tpt, n, want, &tl.fin_words, &tl.aux_bytes);
                if (!P.stage_want && tl.aux_bytes < need) plant_smem_split(tpt, n, 0, &tl.fin_words, &tl.aux_bytes);
            }
            tl.fin_bits = tl.fin_words * 32 < n ? tl.fin_words * 32 : n;
            tl.stage_bytes = P.stage_want ? tl.aux_bytes : 0;
            if (small) tl.nwin = P.nwin_sm;
        }
        // the batched form first writes the labels of the phase's trivial
        // roots and lists the others: room for one record per root
        const bool split = first && o.mode == 0 && pe > pb && !from_filler;
        if (split && cap < T + (pe - pb)) {
            uint64_t ncap = cap;
            while (ncap < T + (pe - pb)) ncap *= 2;
            void *bufs[4] = {b_ov.p, b_oh.p, b_od.p, b_op.p};
            CUDA_TRY(grow_records(bufs, parents ? 4 : 3, T, ncap, s));
            b_ov.p = bufs[0];
            b_oh.p = bufs[1];
            b_od.p = bufs[2];
            b_op.p = bufs[3];
            cap = ncap;
        }
        tl.out_v = (uint32_t *)b_ov.p;
        tl.out_h = (uint32_t *)b_oh.p;
        tl.out_d = (uint32_t *)b_od.p;
        tl.out_p = (uint32_t *)b_op.p;
        tl.out_cap = cap;
        bind_control(tl, ctl);
        tl.failed = (uint32_t *)b_fail.p;
        // reset the control block but keep the running output count
        {
            Control c0{};
            c0.out_count = T;
            CUDA_TRY(cudaMemcpyAsync(ctl, &c0, sizeof(Control), cudaMemcpyHostToDevice, s));
        }
        uint32_t count = 0;
        listed = !first;
        if (first && from_filler) {
            // the filler's split listed this phase's roots and counts them on
            // the device; the filler's claim counter is shared
            CUDA_TRY(cudaStreamWaitEvent(s, fin.ev_split, 0));
            if (small) CUDA_TRY(cudaStreamWaitEvent(s, fin.ev_done, 0));  // another slot layout
            Control *fctl = (Control *)fin.ctl.p;
            tl.root_list = (const uint32_t *)fin.roots.p;
            tl.root_begin = 0;
            tl.count_dev = &fctl->list_n;
            tl.next_root = &fctl->next_root;
            count = pe - pb;  // a bound: the kernel reads the listed count
            listed = true;
            list_h.clear();
        } else if (split) {
            CUDA_TRY(launch_split_trivial(tl, pb, pe - pb, (uint32_t *)b_roots.p, &ctl->list_n, s));
            ++launches;
            CUDA_TRY(cudaMemcpyAsync(&list_n, &ctl->list_n, 4, cudaMemcpyDeviceToHost, s));
            CUDA_TRY(cudaStreamSynchronize(s));
            tl.root_list = (const uint32_t *)b_roots.p;
            tl.root_begin = 0;
            count = list_n;
            listed = true;
            list_h.clear();  // fetched if this attempt fails
        } else if (first) {
            tl.root_list = nullptr;
            tl.root_begin = pb;
            count = pe - pb;
        } else {
            CUDA_TRY(cudaMemcpyAsync(b_roots.p, pending.data(), pending.size() * 4,
                                     cudaMemcpyHostToDevice, s));
            tl.root_list = (const uint32_t *)b_roots.p;
            tl.root_begin = 0;
            count = uint32_t(pending.size());
            list_h = pending;
        }
        tl.root_count = count;
        if (count) {
            if (o.mode == 1) {
                // plain form: one launch per root, one CTA per launch; the claim
                // counter is reset so that launch i builds exactly root i
                for (uint32_t i = 0; i < count; ++i) {
                    TreeLaunch one = tl;
                    if (one.root_list) one.root_list += i; else one.root_begin += i;
                    one.root_count = 1;
                    CUDA_TRY(cudaMemsetAsync(&ctl->next_root, 0, sizeof(unsigned int), s));
                    CUDA_TRY(launch_plant_trees(one, P.tpt, 1, s));
                    ++launches;
                }
            } else if (lt.offsets) {
                // the next phase's first trees fill this launch's tail (see Filler)
                const uint64_t nx = std::min<uint64_t>(
                    std::max<uint64_t>(uint64_t(pe) * 2, uint64_t(pe) + uint64_t(P.slots) * 2), re);
                const bool filler = overlap && first && !small && use_lt && pe < re;
                Filler &fo = fill[ph & 1];
                if (filler) {
                    if (!s2) {
                        CUDA_TRY(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
                        for (Filler &f : fill) {
                            CUDA_TRY(cudaEventCreateWithFlags(&f.ev_clear, cudaEventDisableTiming));
                            CUDA_TRY(cudaEventCreateWithFlags(&f.ev_split, cudaEventDisableTiming));
                            CUDA_TRY(cudaEventCreateWithFlags(&f.ev_done, cudaEventDisableTiming));
                        }
                    }
                    if (!fo.ctl.p) {
                        fo.ctl.s = fo.fail.s = fo.roots.s = fo.ov.s = fo.oh.s = fo.od.s = fo.op.s = fo.stop.s = s;
                        fo.roots_cap = re - rb + 1;
                        // labels of the trees that fit: a tree that does not fit is built again later
                        fo.cap = std::min<uint64_t>(cap, uint64_t(32) << 20) + fo.roots_cap;
                        CUDA_TRY(dmalloc(&fo.ctl.p, sizeof(Control), s));
                        CUDA_TRY(dmalloc(&fo.fail.p, size_t(fo.roots_cap) * 4, s));
                        CUDA_TRY(dmalloc(&fo.roots.p, size_t(fo.roots_cap) * 4, s));
                        CUDA_TRY(dmalloc(&fo.ov.p, fo.cap * 4, s));
                        CUDA_TRY(dmalloc(&fo.oh.p, fo.cap * 4, s));
                        CUDA_TRY(dmalloc(&fo.od.p, fo.cap * 4, s));
                        if (parents) CUDA_TRY(dmalloc(&fo.op.p, fo.cap * 4, s));
                        CUDA_TRY(dmalloc(&fo.stop.p, sizeof(int), s));
                    }
                    CUDA_TRY(cudaMemsetAsync(fo.stop.p, 0, sizeof(int), s));
                    CUDA_TRY(cudaMemsetAsync(fo.ctl.p, 0, sizeof(Control), s));
                    CUDA_TRY(cudaEventRecord(fo.ev_clear, s));
                }
                CUDA_TRY(launch_plant_trees(tl, small ? P.tpt_sm : P.tpt_lt, small ? P.slots_sm : P.slots_lt, s));
                ++launches;
                if (filler) {
                    // stop claiming once this launch is done (ordered after it on s)
                    CUDA_TRY(cudaMemsetAsync(fo.stop.p, 1, sizeof(int), s));
                    Control *fctl = (Control *)fo.ctl.p;
                    TreeLaunch tf = tl;  // this phase's table and launch shape
                    tf.out_v = (uint32_t *)fo.ov.p;
                    tf.out_h = (uint32_t *)fo.oh.p;
                    tf.out_d = (uint32_t *)fo.od.p;
                    tf.out_p = (uint32_t *)fo.op.p;
                    tf.out_cap = fo.cap;
                    bind_control(tf, fctl);
                    tf.failed = (uint32_t *)fo.fail.p;
                    tf.stop = (const int *)fo.stop.p;
                    CUDA_TRY(cudaStreamWaitEvent(s2, fo.ev_clear, 0));
                    CUDA_TRY(launch_split_trivial(tf, pe, uint32_t(nx - pe), (uint32_t *)fo.roots.p,
                                                  &fctl->list_n, s2));
                    CUDA_TRY(cudaEventRecord(fo.ev_split, s2));
                    tf.root_list = (const uint32_t *)fo.roots.p;
                    tf.root_begin = 0;
                    tf.root_count = uint32_t(nx - pe);
                    tf.count_dev = &fctl->list_n;
                    CUDA_TRY(launch_plant_trees(tf, P.tpt_lt, P.slots_lt, s2));
                    CUDA_TRY(cudaEventRecord(fo.ev_done, s2));
                    launches += 2;
                    fo.active = true;
                    fo.pb = pe;
                    fo.pe = uint32_t(nx);
                }
            } else {
                CUDA_TRY(launch_plant_trees(tl, P.tpt, P.slots, s));
                ++launches;
            }
        }
        CUDA_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < 7; ++k) agg[k] += hc.stats[k];
        if (hc.flags[0] == ERR_DIST_OVERFLOW) {
            st = set_error(CHL_EOVERFLOW, "a shortest distance reaches UINT32_MAX");
            goto done;
        }
        if (hc.flags[0] == ERR_ROUND_LIMIT) {
            st = set_error(CHL_ETIMEOUT, "a tree exceeded its round limit");
            goto done;
        }
        if (hc.flags[0] == ERR_WAIT_LIMIT) {
            st = set_error(CHL_ETIMEOUT, "a tree's staging copies did not complete in time");
            goto done;
        }
        T = records_kept(hc);
        std::vector<uint32_t> ffailed;  // the filler's trees that did not fit its buffer
        if (first && from_filler && !filler_merged) {
            // the filler's trees are this phase's too: wait for them, then take
            // their statistics, append their labels after this launch's, and
            // count the shared claim counter and root list as this attempt's
            CUDA_TRY(cudaEventSynchronize(fin.ev_done));
            CUDA_TRY(cudaMemcpy(&fin.hc, fin.ctl.p, sizeof(Control), cudaMemcpyDeviceToHost));
            for (int k = 0; k < 7; ++k) agg[k] += fin.hc.stats[k];
            overlapped += fin.hc.stats[3] - fin.hc.failed_count;
            if (fin.hc.flags[0] == ERR_DIST_OVERFLOW) {
                st = set_error(CHL_EOVERFLOW, "a shortest distance reaches UINT32_MAX");
                goto done;
            }
            if (fin.hc.flags[0]) {
                st = set_error(CHL_ETIMEOUT, "a tree exceeded its round limit or a staging wait (code %d)",
                               fin.hc.flags[0]);
                goto done;
            }
            const uint64_t Tf = records_kept(fin.hc);
            if (Tf) {
                if (cap < T + Tf) {
                    uint64_t ncap = cap;
                    while (ncap < T + Tf) ncap *= 2;
                    void *bufs[4] = {b_ov.p, b_oh.p, b_od.p, b_op.p};
                    CUDA_TRY(grow_records(bufs, parents ? 4 : 3, T, ncap, s));
                    b_ov.p = bufs[0];
                    b_oh.p = bufs[1];
                    b_od.p = bufs[2];
                    b_op.p = bufs[3];
                    cap = ncap;
                }
                CUDA_TRY(cudaMemcpyAsync((uint32_t *)b_ov.p + T, fin.ov.p, Tf * 4, cudaMemcpyDeviceToDevice, s));
                CUDA_TRY(cudaMemcpyAsync((uint32_t *)b_oh.p + T, fin.oh.p, Tf * 4, cudaMemcpyDeviceToDevice, s));
                CUDA_TRY(cudaMemcpyAsync((uint32_t *)b_od.p + T, fin.od.p, Tf * 4, cudaMemcpyDeviceToDevice, s));
                if (parents)
                    CUDA_TRY(cudaMemcpyAsync((uint32_t *)b_op.p + T, fin.op.p, Tf * 4, cudaMemcpyDeviceToDevice, s));
                T += Tf;
            }
            ffailed.resize(fin.hc.failed_count);
            if (!ffailed.empty())
                CUDA_TRY(cudaMemcpy(ffailed.data(), fin.fail.p, ffailed.size() * 4, cudaMemcpyDeviceToHost));
            hc.next_root = fin.hc.next_root;
            count = fin.hc.list_n;
            filler_merged = true;
            fin.active = false;
            free_table(fin.old, s);
        }
        if (!hc.flags[1] && ffailed.empty()) break;  // every root of this attempt fit
        // collect roots that failed or were never claimed, grow the buffer, go again
        {
            std::vector<uint32_t> failed(hc.failed_count);
            if (hc.failed_count)
                CUDA_TRY(cudaMemcpyAsync(failed.data(), b_fail.p, size_t(hc.failed_count) * 4,
                                         cudaMemcpyDeviceToHost, s));
            failed.insert(failed.end(), ffailed.begin(), ffailed.end());
            if (split) {
                list_h.resize(count);
                if (count)
                    CUDA_TRY(cudaMemcpyAsync(list_h.data(), b_roots.p, size_t(count) * 4,
                                             cudaMemcpyDeviceToHost, s));
            } else if (filler_merged && first) {
                list_h.resize(count);
                if (count)
                    CUDA_TRY(cudaMemcpyAsync(list_h.data(), fin.roots.p, size_t(count) * 4,
                                             cudaMemcpyDeviceToHost, s));
            }
            CUDA_TRY(cudaStreamSynchronize(s));
            auto root_at = [&](uint32_t i) { return listed ? list_h[i] : pb + i; };
            claimed_upto = hc.next_root < count ? hc.next_root : count;
            if (o.mode == 1) {
                // launches after the first failure claimed nothing: resume after it
                claimed_upto = count;
                if (!failed.empty()) {
                    for (uint32_t i = 0; i < count; ++i)
                        if (root_at(i) == failed[0]) { claimed_upto = i + 1; break; }
                }
            }
            pending = failed;
            for (uint32_t i = claimed_upto; i < count; ++i) pending.push_back(root_at(i));
            first = false;
            if (attempt > 40) {
                st = set_error(CHL_ENOMEM, "label buffer cannot grow further");
                goto done;
            }
            void *bufs[4] = {b_ov.p, b_oh.p, b_od.p, b_op.p};
            CUDA_TRY(grow_records(bufs, parents ? 4 : 3, T, cap * 2, s));
            b_ov.p = bufs[0];
            b_oh.p = bufs[1];
            b_od.p = bufs[2];
            b_op.p = bufs[3];
            cap *= 2;
        }
    }
    // The switch of Sec. 5.2: label pruning starts once a phase's trees explore
    // many vertices per label (Psi = expansions / labels above psi_th), or once
    // the Common Label Table pruned a large share of their expansions; before
    // that, the per-vertex table query would cost more than it saves.
    if (hybrid && !use_lt && T > T0) {
        const double psi = double(agg[0] - exp0) / double(T - T0);
        const double cut = agg[0] > exp0 ? double(agg[6] - pr0) / double(agg[0] - exp0) : 0.0;
        const double ratio = m2 ? double(T) / double(m2) : 0.0;
        const double ratio_th = o.switch_ratio > 0.0f ? double(o.switch_ratio) : SWITCH_RATIO;
        if (psi > psi_th || (P.eta && cut >= CLT_PRUNE_TH && o.psi_threshold == 0.0f)) use_lt = true;
        else if (ph == 0 && o.psi_threshold == 0.0f && o.switch_ratio >= 0.0f && ratio < ratio_th)
            use_lt = true;
        // far down the ranking and still cheap trees: the rest is one phase
        else if (pe >= std::max<uint64_t>(uint64_t(P.slots) * 8, 8192) && psi < psi_th / 2)
            hybrid_off = true;
    }
    // The small-tree switch: once a label-pruned phase's trees averaged fewer
    // than small_exp expansions (trees only shrink further down the ranking),
    // the later phases run more, smaller blocks per SM, which hides the
    // per-tree latency of start, rounds and emission.
    if (hybrid && ph_lt && !small && o.mode == 0) {
        const uint64_t built = (agg[3] - tr0) - (agg[2] - triv0);
        if (built && double(agg[0] - exp0) / double(built) < double(P.small_exp)) small = true;
    }
    // the bucket-width switch: the next label-pruned phase's trees are big
    // when this phase's averaged BIG_TREE_COVER of the vertices
    {
        const uint64_t built = (agg[3] - tr0) - (agg[2] - triv0);
        big = built && double(agg[0] - exp0) / double(built) >= BIG_TREE_COVER * double(n);
    }
    if (hybrid && !table.buf.p) {
        // the first phase built the table's trees: the Common Label Table from
        // their labels, for every later phase
        CUDA_TRY(cudaEventRecord(ev[5], s));
        st = table_from_records(rg, P, (const uint32_t *)b_ov.p, (const uint32_t *)b_oh.p,
                                (const uint32_t *)b_od.p, T, s, table, &launches);
        if (st != CHL_OK) goto done;
        CUDA_TRY(cudaEventRecord(ev[6], s));
        with_table = true;
    }
    // The next phase is one more wave of trees after the first (the table's
    // pruning share decides the switch), doubles while the label table is
    // used, so that it stays fresh, and grows fourfold before; after a phase
    // that ran the small-tree launch, it grows fourfold again (those trees are
    // tiny: a phase's fixed cost of table growth and host round trip outweighs
    // the table's freshness). A phase that did not run it doubles, which the
    // next phase's overlapped first trees (launched during it) rely on.
    if (hybrid && pe < re) {
        const uint64_t step_min = uint64_t(P.slots) * 2;
        const uint64_t nx = hybrid_off ? re
                            : ph == 0 ? uint64_t(pe) + P.slots
                                      : std::max<uint64_t>(uint64_t(pe) * (use_lt && !ph_small ? 2 : 4), pe + step_min);
        phases.push_back({pe, uint32_t(std::min<uint64_t>(nx, re))});
    }
    double t_tree = trace ? now_ms() - t_ph : 0;
    if (use_lt && ph + 1 < phases.size()) {
        // every label so far, as CSR, for the next phase's pruning: the first
        // time sorted from all records, then grown by each phase's new ones
        if (!b_ltroot.p) {
            const size_t ls = size_t(std::max(P.slots_lt, P.slots_sm));
            CUDA_TRY(dmalloc(&b_ltroot.p, ls * n * 4, s));
            CUDA_TRY(cudaMemsetAsync(b_ltroot.p, 0xFF, ls * n * 4, s));
        }
        // hubs of the Common Label Table are left out: every tree of a label-
        // pruned phase also queries that table, which holds all their labels
        const uint32_t min_hub = table.buf.p ? table.hubs : 0;
        if (!lt.offsets)
            CUDA_TRY(assemble_table(n, T, (const uint32_t *)b_ov.p, (const uint32_t *)b_oh.p,
                                    (const uint32_t *)b_od.p, rg.pos_of, min_hub, lt, s, &launches));
        else
            CUDA_TRY(grow_table(n, lt, lt_records, T, (const uint32_t *)b_ov.p,
                                (const uint32_t *)b_oh.p, (const uint32_t *)b_od.p, rg.pos_of, min_hub,
                                s, &launches, fill[ph & 1].active ? &fill[ph & 1].old : nullptr));
        lt_records = T;
    }
    if (trace) {
        CUDA_TRY(cudaStreamSynchronize(s));
        std::fprintf(stderr,
                     "chl phase %zu roots [%u, %u) table %d%s%s trees %.3f ms assemble %.3f ms "
                     "expanded %llu arcs %llu labels %llu rounds %llu buckets %llu pruned %llu\n",
                     ph, pb, pe, ph_lt, ph_small ? " small" : "", ph_narrow ? " narrow" : "", t_tree,
                     now_ms() - t_ph - t_tree,
                     (unsigned long long)(agg[0] - exp0), (unsigned long long)(agg[1] - arc0),
                     (unsigned long long)(T - T0), (unsigned long long)(agg[4] - rd0),
                     (unsigned long long)(agg[5] - bk0), (unsigned long long)(agg[6] - pr0));
    }
    }  // phases
    free_table(lt, s);
    CUDA_TRY(cudaEventRecord(ev[2], s));
    // slot state and table are no longer needed: release them before assembly
    slot.release();
    table.buf.release();
    b_ltroot.release();

    CUDA_TRY(assemble_labels(n, T, (const uint32_t *)b_ov.p, (const uint32_t *)b_oh.p,
                             (const uint32_t *)b_od.p, rg.vert_at, csr, &too_long, s, &launches));
    if (too_long) {
        st = set_error(CHL_EOVERFLOW, "a vertex holds more labels than the segment sorter supports");
        goto done;
    }
    if (parents) {
        CUDA_TRY(dmalloc(&csr_parent, (T ? T : 1) * 4, s));
        CUDA_TRY(place_parents(T, (const uint32_t *)b_ov.p, (const uint32_t *)b_oh.p,
                               (const uint32_t *)b_op.p, csr, csr_parent, s, &launches));
    }
    CUDA_TRY(cudaEventRecord(ev[3], s));
    CUDA_TRY(cudaEventSynchronize(ev[3]));
    cudaEventElapsedTime(&ms_total, ev[0], ev[3]);
    cudaEventElapsedTime(&ms_tree, ev[1], ev[2]);
    cudaEventElapsedTime(&ms_sort, ev[2], ev[3]);
    if (trace) {
        float ms_prep = 0;
        cudaEventElapsedTime(&ms_prep, ev[0], ev[1]);
        std::fprintf(stderr, "chl build total %.3f ms: inputs, checks and buffers %.3f ms, phases %.3f ms, "
                     "label sort %.3f ms\n", ms_total, ms_prep, ms_tree, ms_sort);
    }
    if (with_table && hybrid) cudaEventElapsedTime(&ms_table, ev[5], ev[6]);
    else if (with_table) cudaEventElapsedTime(&ms_table, ev[1], ev[4]);

    L = new (std::nothrow) chl_labels;
    if (!L) {
        st = set_error(CHL_ENOMEM, "host allocation failed");
        goto done;
    }
    L->n = n;
    L->total = T;
    L->offsets = csr.offsets;
    L->hub = csr.hub;
    L->hubpos = csr.hubpos;
    L->dist = csr.dist;
    L->parent = csr_parent;
    csr_parent = nullptr;
    L->bytes = (uint64_t(n) + 1) * 8 + T * (L->parent ? 16 : 12);
    L->device = dev;
    L->stats.trees = agg[3];
    L->stats.labels = T;
    L->stats.expanded = agg[0];
    L->stats.arcs = agg[1];
    L->stats.trivial = agg[2];
    L->stats.rounds = agg[4];
    L->stats.buckets = agg[5];
    L->stats.pruned = agg[6];
    L->stats.build_ms = ms_total;
    L->stats.tree_ms = ms_tree;
    L->stats.sort_ms = ms_sort;
    L->stats.table_ms = ms_table;
    L->stats.phases = phases.size();
    L->stats.label_table_phases = lt_phases;
    L->stats.small_tree_phases = small_phases;
    L->stats.overlapped_trees = overlapped;
    L->stats.launches = uint64_t(launches);
    csr = LabelCSR{};
    *out = L;
done:
    if (s2) {
        // the fillers' trees read buffers freed below on s
        cudaStreamSynchronize(s2);
        cudaStreamDestroy(s2);
    }
    for (Filler &f : fill) {
        free_table(f.old, s);
        for (cudaEvent_t e : {f.ev_clear, f.ev_split, f.ev_done})
            if (e) cudaEventDestroy(e);
    }
    free_table(lt, s);
    if (csr_parent) cudaFreeAsync(csr_parent, s);
    if (csr.offsets) cudaFreeAsync(csr.offsets, s);
    if (csr.hub) cudaFreeAsync(csr.hub, s);
    if (csr.hubpos) cudaFreeAsync(csr.hubpos, s);
    if (csr.dist) cudaFreeAsync(csr.dist, s);
    free_graph(rg, s);
    for (auto &e : ev)
        if (e) cudaEventDestroy(e);
    // DevBuf destructors release the rest on stream s
    return st;
}

extern "C" chl_status chl_labels_info(const chl_labels *L, uint32_t *n, uint64_t *total,
                                      uint64_t *bytes) {
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    if (n) *n = L->n;
    if (total) *total = L->total;
    if (bytes) *bytes = L->bytes;
    return CHL_OK;
}

extern "C" chl_status chl_labels_stats(const chl_labels *L, chl_build_stats *stats) {
    if (!L || !stats) return set_error(CHL_EINVAL, "NULL argument");
    *stats = L->stats;
    return CHL_OK;
}

extern "C" chl_status chl_labels_view(const chl_labels *L, const uint64_t **offsets,
                                      const uint32_t **hub, const uint32_t **dist) {
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    if (offsets) *offsets = L->offsets;
    if (hub) *hub = L->hub;
    if (dist) *dist = L->dist;
    return CHL_OK;
}

extern "C" chl_status chl_labels_copy(const chl_labels *L, uint64_t *offsets, uint32_t *hub,
                                      uint32_t *dist, chl_mem dst_mem, void *stream) {
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    if (dst_mem != CHL_MEM_DEVICE && dst_mem != CHL_MEM_HOST)
        return set_error(CHL_EINVAL, "unknown memory kind");
    CHECK_DEVICE(L);
    cudaStream_t s = (cudaStream_t)stream;
    const cudaMemcpyKind k = dst_mem == CHL_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    chl_status st = CHL_OK;
    if (offsets) CUDA_TRY(cudaMemcpyAsync(offsets, L->offsets, (size_t(L->n) + 1) * 8, k, s));
    if (hub && L->total) CUDA_TRY(cudaMemcpyAsync(hub, L->hub, L->total * 4, k, s));
    if (dist && L->total) CUDA_TRY(cudaMemcpyAsync(dist, L->dist, L->total * 4, k, s));
    CUDA_TRY(cudaStreamSynchronize(s));
done:
    return st;
}

extern "C" chl_status chl_query(const chl_labels *L, const uint32_t *pairs, uint64_t q,
                                uint32_t *out, chl_mem mem, void *stream) {
    ENTER();
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    CHECK_DEVICE(L);
    if (q == 0) return CHL_OK;
    if (!pairs || !out) return set_error(CHL_EINVAL, "pairs or out is NULL");
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    DevBuf b_p, b_o, b_bad;
    b_p.s = b_o.s = b_bad.s = s;
    const uint32_t *dp = pairs;
    uint32_t *dout = out;
    int hbad = 0;
    CUDA_TRY(dmalloc(&b_bad.p, sizeof(int), s));
    CUDA_TRY(cudaMemsetAsync(b_bad.p, 0, sizeof(int), s));
    if (mem == CHL_MEM_HOST) {
        CUDA_TRY(dmalloc(&b_p.p, q * 8, s));
        CUDA_TRY(dmalloc(&b_o.p, q * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_p.p, pairs, q * 8, cudaMemcpyHostToDevice, s));
        dp = (const uint32_t *)b_p.p;
        dout = (uint32_t *)b_o.p;
    }
    CUDA_TRY(launch_query(L->n, L->offsets, L->hubpos, L->dist, dp, q, dout, (int *)b_bad.p, s));
    if (mem == CHL_MEM_HOST) CUDA_TRY(cudaMemcpyAsync(out, dout, q * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hbad, b_bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) st = set_error(CHL_EINVAL, "a query vertex id is >= n");
done:
    return st;
}

// ------------------------------------------------------------------ query modes
namespace {

// a batch over one set (plain or partitioned) through the multi-set kernel:
// device pairs and answers, the set descriptor and a flag in device memory
chl_status run_set_query(const QuerySet &set, const QuerySet *parts_h, uint32_t nparts,
                         const uint32_t *pairs, uint64_t q, uint32_t *out, chl_mem mem, bool grouped,
                         cudaStream_t s) {
    chl_status st = CHL_OK;
    DevBuf b_set, b_p, b_o, b_perm, b_scr;
    b_set.s = b_p.s = b_o.s = b_perm.s = b_scr.s = s;
    const uint32_t *dp = pairs;
    uint32_t *dout = out;
    int hbad = 0;
    // [set][nsets, bad][parts]
    const size_t hdr = sizeof(QuerySet) + 16;
    std::vector<uint8_t> host(hdr + size_t(nparts) * sizeof(QuerySet));
    QuerySet top = set;
    uint8_t *base = nullptr;
    CUDA_TRY(dmalloc(&b_set.p, host.size(), s));
    base = static_cast<uint8_t *>(b_set.p);
    if (nparts) top.parts = reinterpret_cast<const QuerySet *>(base + hdr);
    std::memcpy(host.data(), &top, sizeof(QuerySet));
    {
        const uint32_t one = 1, zero = 0;
        std::memcpy(host.data() + sizeof(QuerySet), &one, 4);
        std::memcpy(host.data() + sizeof(QuerySet) + 4, &zero, 4);
    }
    if (nparts) std::memcpy(host.data() + hdr, parts_h, size_t(nparts) * sizeof(QuerySet));
    CUDA_TRY(cudaMemcpyAsync(base, host.data(), host.size(), cudaMemcpyHostToDevice, s));
    if (mem == CHL_MEM_HOST) {
        CUDA_TRY(dmalloc(&b_p.p, q * 8, s));
        CUDA_TRY(dmalloc(&b_o.p, q * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_p.p, pairs, q * 8, cudaMemcpyHostToDevice, s));
        dp = (const uint32_t *)b_p.p;
        dout = (uint32_t *)b_o.p;
    }
    if (grouped) {
        CUDA_TRY(dmalloc(&b_perm.p, q * 4, s));
        CUDA_TRY(dmalloc(&b_scr.p, GROUP_SCRATCH_WORDS * 4, s));
        CUDA_TRY(launch_group_order(reinterpret_cast<const QuerySet *>(base),
                                    reinterpret_cast<const uint32_t *>(base + sizeof(QuerySet)), dp,
                                    nullptr, q, (uint32_t *)b_scr.p, (uint32_t *)b_perm.p, s));
    }
    CUDA_TRY(launch_query_sets(reinterpret_cast<const QuerySet *>(base),
                               reinterpret_cast<const uint32_t *>(base + sizeof(QuerySet)), dp, nullptr,
                               grouped ? (const uint32_t *)b_perm.p : nullptr, q, dout,
                               reinterpret_cast<int *>(base + sizeof(QuerySet) + 4), device_sms() * 64, s));
    if (mem == CHL_MEM_HOST) CUDA_TRY(cudaMemcpyAsync(out, dout, q * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hbad, base + sizeof(QuerySet) + 4, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) st = set_error(CHL_EINVAL, "a query vertex id is >= n");
done:
    return st;
}

}  // namespace

extern "C" chl_status chl_query_partitioned(const chl_labels *const *parts, uint32_t nparts,
                                            const uint32_t *pairs, uint64_t q, uint32_t *out, chl_mem mem,
                                            void *stream) {
    ENTER();
    if (!parts) return set_error(CHL_EINVAL, "parts is NULL");
    if (nparts < 1 || nparts > CHL_MAX_PARTS)
        return set_error(CHL_EINVAL, "nparts must be in [1, %d]", CHL_MAX_PARTS);
    std::vector<QuerySet> h(nparts);
    for (uint32_t k = 0; k < nparts; ++k) {
        if (!parts[k]) return set_error(CHL_EINVAL, "part %u is NULL", k);
        CHECK_DEVICE(parts[k]);
        if (parts[k]->n != parts[0]->n) return set_error(CHL_EINVAL, "parts cover different vertex counts");
        h[k] = QuerySet{parts[k]->n, parts[k]->offsets, parts[k]->hubpos, parts[k]->dist, 0, nullptr};
    }
    if (q == 0) return CHL_OK;
    if (!pairs || !out) return set_error(CHL_EINVAL, "pairs or out is NULL");
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    const QuerySet set{parts[0]->n, nullptr, nullptr, nullptr, nparts, nullptr};
    return run_set_query(set, h.data(), nparts, pairs, q, out, mem, false, (cudaStream_t)stream);
}

extern "C" chl_status chl_query_grouped(const chl_labels *L, const uint32_t *pairs, uint64_t q,
                                        uint32_t *out, chl_mem mem, void *stream) {
    ENTER();
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    CHECK_DEVICE(L);
    if (q == 0) return CHL_OK;
    if (!pairs || !out) return set_error(CHL_EINVAL, "pairs or out is NULL");
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    if (q > 0xFFFFFFFFull) return set_error(CHL_EINVAL, "chl_query_grouped takes fewer than 2^32 pairs");
    const QuerySet set{L->n, L->offsets, L->hubpos, L->dist, 0, nullptr};
    return run_set_query(set, nullptr, 0, pairs, q, out, mem, true, (cudaStream_t)stream);
}

extern "C" void chl_labels_free(chl_labels *L) {
    if (!L) return;
    // free on the device that holds the arrays, then restore the caller's
    int cur = -1;
    const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != L->device;
    if (other) cudaSetDevice(L->device);
    cudaFree(L->offsets);
    cudaFree(L->hub);
    cudaFree(L->hubpos);
    cudaFree(L->dist);
    if (L->parent) cudaFree(L->parent);
    if (other) cudaSetDevice(cur);
    delete L;
}

extern "C" chl_status chl_labels_parents(const chl_labels *L, uint32_t *parent, chl_mem mem,
                                         void *stream) {
    ENTER();
    if (!L || !parent) return set_error(CHL_EINVAL, "labels or parent is NULL");
    if (!L->parent) return set_error(CHL_EINVAL, "labels were built without CHL_FLAG_PARENTS");
    CHECK_DEVICE(L);
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    if (L->total) {
        CUDA_TRY(cudaMemcpyAsync(parent, L->parent, L->total * 4,
                                 mem == CHL_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
done:
    return st;
}

extern "C" chl_status chl_path(const chl_labels *L, const uint32_t *pairs, uint64_t q, uint32_t max_len,
                               uint32_t *paths, uint32_t *lens, chl_mem mem, void *stream) {
    ENTER();
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    if (!L->parent) return set_error(CHL_EINVAL, "labels were built without CHL_FLAG_PARENTS");
    CHECK_DEVICE(L);
    if (q == 0) return CHL_OK;
    if (!pairs || !lens || (max_len && !paths)) return set_error(CHL_EINVAL, "NULL argument");
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    DevBuf b_p, b_path, b_len, b_bad;
    b_p.s = b_path.s = b_len.s = b_bad.s = s;
    const uint32_t *dp = pairs;
    uint32_t *dpath = paths, *dlen = lens;
    int hbad = 0;
    CUDA_TRY(dmalloc(&b_bad.p, sizeof(int), s));
    CUDA_TRY(cudaMemsetAsync(b_bad.p, 0, sizeof(int), s));
    if (mem == CHL_MEM_HOST) {
        CUDA_TRY(dmalloc(&b_p.p, q * 8, s));
        CUDA_TRY(dmalloc(&b_path.p, q * max_len * 4 + 4, s));
        CUDA_TRY(dmalloc(&b_len.p, q * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_p.p, pairs, q * 8, cudaMemcpyHostToDevice, s));
        dp = (const uint32_t *)b_p.p;
        dpath = (uint32_t *)b_path.p;
        dlen = (uint32_t *)b_len.p;
    }
    CUDA_TRY(launch_paths(L->n, L->offsets, L->hubpos, L->dist, L->hub, L->parent, dp, q, max_len,
                          dpath, dlen, (int *)b_bad.p, s));
    if (mem == CHL_MEM_HOST) {
        if (max_len) CUDA_TRY(cudaMemcpyAsync(paths, dpath, q * max_len * 4, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaMemcpyAsync(lens, dlen, q * 4, cudaMemcpyDeviceToHost, s));
    }
    CUDA_TRY(cudaMemcpyAsync(&hbad, b_bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad == 1) st = set_error(CHL_EINVAL, "a query vertex id is >= n");
    else if (hbad) st = set_error(CHL_ECUDA, "a parent chain did not reach its hub");
done:
    return st;
}

// ------------------------------------------------------------------ queries without allocation
// chl_query_noalloc serves callers that must not allocate device memory at
// query time: a request path running inside a memory budget that another
// runtime owns, or a latency-critical thread that cannot afford the
// allocator's synchronisation. It runs the same query kernel as chl_query
// but stages pairs, answers and the bad-vertex flag in one fixed device
// array of this file instead of memory allocated per call.
namespace {

constexpr uint64_t NOALLOC_MAX_PAIRS = uint64_t(1) << 20;
constexpr int NOALLOC_MAX_DEVICES = 64;

struct NoAllocScratch {
    uint32_t pairs[2 * NOALLOC_MAX_PAIRS];
    uint32_t out[NOALLOC_MAX_PAIRS];
    int bad;
};

// Host code must not use this name as a device address: it is a host-side
// stand-in. Its device address is resolved per device with
// cudaGetSymbolAddress below. Every GPU that loads the library holds it
// (about 12 MiB) until the process exits.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

std::mutex g_noalloc_mu;
NoAllocScratch *g_noalloc_addr[NOALLOC_MAX_DEVICES] = {};

}  // namespace

extern "C" chl_status chl_query_noalloc(const chl_labels *L, const uint32_t *pairs, uint64_t q,
                                        uint32_t *out, chl_mem mem, void *stream) {
    ENTER();
    if (!L) return set_error(CHL_EINVAL, "labels is NULL");
    CHECK_DEVICE(L);
    if (q == 0) return CHL_OK;
    if (!pairs || !out) return set_error(CHL_EINVAL, "pairs or out is NULL");
    if (mem != CHL_MEM_DEVICE && mem != CHL_MEM_HOST) return set_error(CHL_EINVAL, "unknown memory kind");
    if (q > NOALLOC_MAX_PAIRS)
        return set_error(CHL_EINVAL, "chl_query_noalloc takes at most %llu pairs per call, got %llu",
                         (unsigned long long)NOALLOC_MAX_PAIRS, (unsigned long long)q);
    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    int dev = 0, hbad = 0;
    NoAllocScratch *sc = nullptr;
    const uint32_t *dp = pairs;
    uint32_t *dout = out;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        st = set_error(CHL_EINVAL, "device %d outside the %d devices supported", dev, NOALLOC_MAX_DEVICES);
        goto done;
    }
    {
        // first call on a device: resolve the scratch array's device address
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_addr[dev]) {
            void *a = nullptr;
            CUDA_TRY(cudaGetSymbolAddress(&a, g_noalloc_scratch));
            g_noalloc_addr[dev] = (NoAllocScratch *)a;
        }
        sc = g_noalloc_addr[dev];
    }
    CUDA_TRY(cudaMemsetAsync(&sc->bad, 0, sizeof(int), s));
    if (mem == CHL_MEM_HOST) {
        CUDA_TRY(cudaMemcpyAsync(sc->pairs, pairs, q * 8, cudaMemcpyHostToDevice, s));
        dp = sc->pairs;
        dout = sc->out;
    }
    CUDA_TRY(launch_query(L->n, L->offsets, L->hubpos, L->dist, dp, q, dout, &sc->bad, s));
    if (mem == CHL_MEM_HOST) CUDA_TRY(cudaMemcpyAsync(out, sc->out, q * 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(&hbad, &sc->bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) st = set_error(CHL_EINVAL, "a query vertex id is >= n");
done:
    return st;
}

// ------------------------------------------------------------------ autotuner
namespace {

// One trial: the tree kernel alone on a root list, with fresh slot state;
// returns its device time (ms) or a negative value when the labels did not
// fit the trial buffer.
chl_status tree_trial(const RankGraph &rg, const Params &P, const CommonTable &table,
                      const uint32_t *roots, uint32_t count, uint64_t cap, cudaStream_t s, float *ms,
                      unsigned long long *stats4) {
    chl_status st = CHL_OK;
    const uint32_t n = rg.n;
    DevBuf b_ctl, b_ov, b_oh, b_od, b_fail;
    SlotState slot;
    b_ctl.s = b_ov.s = b_oh.s = b_od.s = b_fail.s = s;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    Control hc{};
    Control *ctl = nullptr;
    TreeLaunch tl{};
    *ms = -1.0f;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    CUDA_TRY(slot.alloc(P, n, s));
    CUDA_TRY(dmalloc(&b_ctl.p, sizeof(Control), s));
    CUDA_TRY(cudaMemsetAsync(b_ctl.p, 0, sizeof(Control), s));
    CUDA_TRY(dmalloc(&b_fail.p, size_t(count + 1) * 4, s));
    CUDA_TRY(dmalloc(&b_ov.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_oh.p, cap * 4, s));
    CUDA_TRY(dmalloc(&b_od.p, cap * 4, s));
    ctl = (Control *)b_ctl.p;
    tl.n = n;
    tl.row = rg.row;
    tl.arc = rg.arc;
    tl.vert_at = rg.vert_at;
    tl.root_list = roots;
    tl.root_begin = 0;
    tl.root_count = count;
    slot.fill(P, n, tl);
    table.fill(tl);
    tl.out_v = (uint32_t *)b_ov.p;
    tl.out_h = (uint32_t *)b_oh.p;
    tl.out_d = (uint32_t *)b_od.p;
    tl.out_cap = cap;
    bind_control(tl, ctl);
    tl.failed = (uint32_t *)b_fail.p;
    CUDA_TRY(cudaEventRecord(e0, s));
    CUDA_TRY(launch_plant_trees(tl, P.tpt, P.slots, s));
    CUDA_TRY(cudaEventRecord(e1, s));
    CUDA_TRY(cudaMemcpyAsync(&hc, ctl, sizeof(Control), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (hc.flags[0]) {
        st = set_error(hc.flags[0] == ERR_DIST_OVERFLOW ? CHL_EOVERFLOW : CHL_ETIMEOUT,
                       "tuning trial failed (code %d)", hc.flags[0]);
        goto done;
    }
    if (!hc.flags[1]) CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    for (int k = 0; k < 4; ++k) stats4[k] = hc.stats[k];
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

}  // namespace

extern "C" chl_status chl_tune(const chl_csr *g, const uint32_t *rank, const chl_build_opts *base,
                               void *stream, chl_build_opts *best, chl_tune_report *report) {
    ENTER();
    if (!g || !rank || !best) return set_error(CHL_EINVAL, "graph, rank or best is NULL");
    if (g->n == 0) return set_error(CHL_EINVAL, "graph has no vertices");
    if (g->n >= 0x7FFFFFFFu) return set_error(CHL_EINVAL, "n must be < 2^31");
    if (!g->row_ptr || (g->num_arcs && (!g->col || !g->w)))
        return set_error(CHL_EINVAL, "graph arrays are NULL");
    if (g->mem != CHL_MEM_DEVICE && g->mem != CHL_MEM_HOST)
        return set_error(CHL_EINVAL, "unknown memory kind");
    chl_build_opts o{};
    if (base) o = *base;
    if (o.mode != 0) return set_error(CHL_EINVAL, "chl_tune tunes the batched mode (mode 0)");
    if (o.common_hubs > int32_t(CHL_MAX_COMMON_HUBS))
        return set_error(CHL_EINVAL, "common_hubs must be at most %d", CHL_MAX_COMMON_HUBS);
    if (o.flags & ~int32_t(CHL_FLAG_WIDE_KEYS | CHL_FLAG_PARENTS | CHL_FLAG_NO_HYBRID |
                           CHL_FLAG_DENSE_ROOT_LABELS))
        return set_error(CHL_EINVAL, "unknown bit in flags");
    cudaStream_t s = (cudaStream_t)stream;
    chl_status st = CHL_OK;
    const uint32_t n = g->n;
    const uint64_t m2 = g->num_arcs;
    const uint64_t *d_row = g->row_ptr;
    const uint32_t *d_col = g->col, *d_w = g->w, *d_rank = rank;
    DevBuf b_row, b_col, b_w, b_rank, b_roots;
    CommonTable table;
    b_row.s = b_col.s = b_w.s = b_rank.s = b_roots.s = s;
    RankGraph rg;
    int launches = 0, dev = 0, sms = 0, trials = 0;
    size_t free_b = 0, total_b = 0;
    std::vector<uint32_t> roots;
    uint32_t K = 0;
    uint64_t cap = 0;
    Params bestP{};
    float best_ms = -1.0f;
    unsigned long long best_stats[4] = {0, 0, 0, 0};
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (g->mem == CHL_MEM_HOST) {
        CUDA_TRY(dmalloc(&b_row.p, (size_t(n) + 1) * 8, s));
        CUDA_TRY(dmalloc(&b_col.p, (m2 ? m2 : 1) * 4, s));
        CUDA_TRY(dmalloc(&b_w.p, (m2 ? m2 : 1) * 4, s));
        CUDA_TRY(dmalloc(&b_rank.p, size_t(n) * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_row.p, g->row_ptr, (size_t(n) + 1) * 8, cudaMemcpyHostToDevice, s));
        if (m2) {
            CUDA_TRY(cudaMemcpyAsync(b_col.p, g->col, m2 * 4, cudaMemcpyHostToDevice, s));
            CUDA_TRY(cudaMemcpyAsync(b_w.p, g->w, m2 * 4, cudaMemcpyHostToDevice, s));
        }
        CUDA_TRY(cudaMemcpyAsync(b_rank.p, rank, size_t(n) * 4, cudaMemcpyHostToDevice, s));
        d_row = (const uint64_t *)b_row.p;
        d_col = (const uint32_t *)b_col.p;
        d_w = (const uint32_t *)b_w.p;
        d_rank = (const uint32_t *)b_rank.p;
    }
    st = prepare_graph(n, m2, d_row, d_col, d_w, d_rank, rg, s, &launches);
    if (st != CHL_OK) goto done;
    CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    {
        // rank-strided sample: every (n/K)-th rank position, about four trees per slot
        const Params p0 = choose_params(rg, o, sms, free_b);
        K = uint32_t(4 * (uint64_t)p0.slots);
        if (K > n) K = n;
        if (K < 1) K = 1;
        roots.resize(K);
        for (uint32_t i = 0; i < K; ++i) roots[i] = uint32_t((uint64_t(i) * n) / K);
        CUDA_TRY(dmalloc(&b_roots.p, size_t(K) * 4, s));
        CUDA_TRY(cudaMemcpyAsync(b_roots.p, roots.data(), size_t(K) * 4, cudaMemcpyHostToDevice, s));
        cap = uint64_t(K) * 256 + 4 * uint64_t(n);
        const uint64_t fit = uint64_t(0.15 * double(free_b)) / 12;
        if (cap > fit) cap = fit;
        // the trials prune with the Common Label Table as the build will
        if (p0.eta && n > p0.eta) {
            SlotState ts;
            CUDA_TRY(ts.alloc(p0, n, s));
            st = build_common_table(rg, p0, ts, s, table, &launches, nullptr);
            if (st != CHL_OK) goto done;
        }
    }
    {
        // coordinate search: bucket width, then threads per tree, then window
        const double wm = rg.w_mean > 1.0 ? rg.w_mean : 1.0;
        std::vector<uint32_t> deltas;
        if (o.bucket_delta > 0) {
            deltas.push_back(uint32_t(o.bucket_delta));
        } else {
            const double f[] = {0.0, 1.0 / 64, 1.0 / 16, 1.0 / 4, 1.0, 2.0};
            for (double x : f) {
                // powers of two: the kernel then finds buckets with a shift
                uint32_t d = 1;
                while (double(d) * 1.5 < wm * x && d < (1u << 30)) d <<= 1;
                bool seen = false;
                for (uint32_t e : deltas) seen |= (e == d);
                if (!seen) deltas.push_back(d);
            }
        }
        std::vector<int> tpts;
        if (o.threads_per_tree) tpts.push_back(o.threads_per_tree);
        else tpts = {256, 128, 512, 1024};
        std::vector<int> wins;
        if (o.window_buckets) wins.push_back(o.window_buckets);
        else wins = {32, 16, 64};
        auto run = [&](uint32_t d, int t, int w, Params *outP, float *outms,
                       unsigned long long *st4) -> chl_status {
            chl_build_opts q = o;
            q.bucket_delta = int32_t(d);
            q.threads_per_tree = t;
            q.window_buckets = w;
            size_t fb = 0, tb = 0;
            cudaMemGetInfo(&fb, &tb);
            Params P = choose_params(rg, q, sms, fb);
            float ms = -1.0f;
            uint64_t c = cap;
            chl_status r = CHL_OK;
            for (int a = 0; a < 4; ++a) {
                r = tree_trial(rg, P, table, (const uint32_t *)b_roots.p, K, c, s, &ms, st4);
                if (r != CHL_OK || ms >= 0) break;
                c *= 4;  // labels did not fit: a larger trial buffer
            }
            ++trials;
            *outP = P;
            *outms = ms;
            return r;
        };
        Params P;
        float ms;
        unsigned long long st4[4];
        for (uint32_t d : deltas) {
            st = run(d, tpts[0], wins[0], &P, &ms, st4);
            if (st != CHL_OK) goto done;
            if (ms >= 0 && (best_ms < 0 || ms < best_ms)) { best_ms = ms; bestP = P; std::copy(st4, st4 + 4, best_stats); }
        }
        for (size_t i = 1; i < tpts.size(); ++i) {
            st = run(bestP.delta, tpts[i], int(bestP.nwin), &P, &ms, st4);
            if (st != CHL_OK) goto done;
            if (ms >= 0 && ms < best_ms) { best_ms = ms; bestP = P; std::copy(st4, st4 + 4, best_stats); }
        }
        for (size_t i = 1; i < wins.size(); ++i) {
            st = run(bestP.delta, bestP.tpt, wins[i], &P, &ms, st4);
            if (st != CHL_OK) goto done;
            if (ms >= 0 && ms < best_ms) { best_ms = ms; bestP = P; std::copy(st4, st4 + 4, best_stats); }
        }
    }
    if (best_ms < 0) {
        st = set_error(CHL_ENOMEM, "no tuning trial completed");
        goto done;
    }
    *best = o;
    best->threads_per_tree = bestP.tpt;
    best->bucket_delta = int32_t(bestP.delta);
    best->window_buckets = int32_t(bestP.nwin);
    best->slots = o.slots;  // 0 keeps the memory-budgeted default at build time
    // A whole build runs in hybrid phases whose pruned trees are far smaller
    // than the sample's: the block size, then the switch points of the phases
    // (the first-phase switch on labels per arc, on or off; the frontier size
    // below which later phases run the small-tree launch; the narrow bucket
    // width after big trees, on or off) are settled by whole builds, one knob
    // at a time.
    if (!o.root_begin && !o.root_end && !(o.flags & CHL_FLAG_NO_HYBRID)) {
        double best_build = -1.0;
        bool pruned_phases = false;  // the last whole build ran label-pruned phases
        auto whole = [&](const chl_build_opts &q, double *ms) -> chl_status {
            chl_labels *Lt = nullptr;
            const chl_status r = chl_build(g, rank, &q, stream, &Lt);
            if (r != CHL_OK) return r;
            *ms = Lt->stats.tree_ms;
            pruned_phases = Lt->stats.label_table_phases > 0;
            chl_labels_free(Lt);
            ++trials;
            return CHL_OK;
        };
        if (!o.threads_per_tree) {
            int best_tpt = bestP.tpt;
            for (int t : {256, 512, 1024}) {
                chl_build_opts q = *best;
                q.threads_per_tree = t;
                double ms = 0;
                if ((st = whole(q, &ms)) != CHL_OK) goto done;
                if (best_build < 0 || ms < best_build) { best_build = ms; best_tpt = t; }
            }
            best->threads_per_tree = best_tpt;
        } else {
            if ((st = whole(*best, &best_build)) != CHL_OK) goto done;
        }
        if (o.switch_ratio == 0.0f && o.psi_threshold == 0.0f) {
            chl_build_opts q = *best;
            q.switch_ratio = -1.0f;  // Psi rule alone
            double ms = 0;
            if ((st = whole(q, &ms)) != CHL_OK) goto done;
            if (ms < best_build) { best_build = ms; best->switch_ratio = -1.0f; }
        }
        if (!o.small_tree_expansions) {
            uint32_t best_small = 0;
            for (uint32_t x : {2048u, 32768u}) {
                chl_build_opts q = *best;
                q.small_tree_expansions = x;
                double ms = 0;
                if ((st = whole(q, &ms)) != CHL_OK) goto done;
                if (ms < best_build) { best_build = ms; best_small = x; }
            }
            best->small_tree_expansions = best_small;
        }
        if (!o.big_tree_bucket_delta) {
            chl_build_opts q = *best;
            q.big_tree_bucket_delta = -1;  // one bucket width for every label-pruned phase
            double ms = 0;
            if ((st = whole(q, &ms)) != CHL_OK) goto done;
            if (ms < best_build) { best_build = ms; best->big_tree_bucket_delta = -1; }
        }
        // The Common Label Table's size (the paper's eta = 16) where the build
        // prunes with the label table too: every hub left out of the dense
        // table is still in the label table, so a smaller one costs a shorter
        // row per expanded vertex and may prune as well
        if (!o.common_hubs) {
            chl_build_opts q = *best;
            double ms = 0;
            if ((st = whole(q, &ms)) != CHL_OK) goto done;
            if (ms < best_build) best_build = ms;
            if (pruned_phases) {
                int best_eta = 0;
                for (int e : {8, 4}) {
                    q.common_hubs = e;
                    if ((st = whole(q, &ms)) != CHL_OK) goto done;
                    if (ms < best_build) { best_build = ms; best_eta = e; }
                }
                best->common_hubs = best_eta;
            }
        }
    }
    if (report) {
        report->trials = trials;
        report->sample_roots = K;
        report->best_tree_ms = best_ms;
        report->best_expanded = best_stats[0];
        report->best_arcs = best_stats[1];
    }
done:
    free_graph(rg, s);
    return st;
}
