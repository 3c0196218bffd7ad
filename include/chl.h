/*
 * chl.h — C ABI of the GB300 canonical hub labeling library (libchl.so).
 *
 * Canonical hub labeling (CHL), Lakhotia et al., "Planting Trees for scalable
 * and efficient Canonical Hub Labeling" (arXiv 1907.00140):
 *
 *   Given an undirected graph G(V,E,W) with positive integer edge weights and
 *   a ranking function R (a total order on V, larger R = more important;
 *   Sec. 1), the CHL holds a label (h, d(v,h)) in L_v exactly when h is the
 *   highest-ranked vertex of SP_{v,h}, the set of vertices on all shortest
 *   v-h paths (Sec. 1; Lemma 1 of Sec. 4.1). It is unique for a fixed R and
 *   minimal (Sec. 1).
 *
 *   chl_build computes it the PLaNT way (Sec. 5.2, Algorithm 3): one
 *   shortest-path tree per root h that carries, for every vertex, its
 *   distance and the highest rank seen on any shortest path to it; a vertex
 *   receives h as a hub when no higher-ranked vertex lies on any of its
 *   shortest paths from h, and a tree stops once every pending vertex is
 *   outranked (early termination, Sec. 5.2). Labels of each vertex are then
 *   sorted by hub rank (Algorithm 2, sort step).
 *
 *   chl_query answers point-to-point shortest distance (PPSD) queries,
 *   d(u,v) = min over common hubs h of d(u,h) + d(v,h) (Sec. 1), by merging
 *   the two rank-sorted label lists (Sec. 6, querying with labels on a single
 *   node).
 *
 * Conventions
 *   - Every function returns a chl_status; no C++ exception crosses the ABI.
 *     On failure chl_last_error() returns a message for the calling thread.
 *   - Pointers marked "device or host" follow the chl_mem value passed with
 *     them: CHL_MEM_DEVICE = CUDA device memory of the current device,
 *     CHL_MEM_HOST = host memory (pinned is faster; pageable works). The
 *     caller keeps ownership of every input and output buffer it passes.
 *   - Work is ordered on the CUDA stream passed as `stream` (a cudaStream_t,
 *     NULL = legacy default stream). A function returns once its results
 *     are complete, unless stated otherwise.
 *   - Distances are uint32; UINT32_MAX means "unreachable". Sums in queries
 *     are taken in 64-bit and saturate at UINT32_MAX.
 *   - The library runs every step on the GPU (sm_103a); it has no CPU
 *     fallback.
 *   - A call that launches work clears the calling thread's CUDA last-error
 *     state (cudaGetLastError) on entry, and again after a CUDA call of its
 *     own failed, so that an error of earlier work is not reported as its
 *     own and a failed allocation does not fail the next call.
 */
#ifndef CHL_H
#define CHL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CHL_OK = 0,
    CHL_EINVAL = 1,     /* malformed argument or input graph / rank */
    CHL_ENOMEM = 2,     /* device or host allocation failed */
    CHL_ECUDA = 3,      /* a CUDA call failed (message holds the CUDA error) */
    CHL_ETIMEOUT = 4,   /* a bounded device wait ran out of iterations */
    CHL_EOVERFLOW = 5   /* a distance reached UINT32_MAX, or a capacity was exceeded */
} chl_status;

typedef enum {
    CHL_MEM_DEVICE = 0,
    CHL_MEM_HOST = 1
} chl_mem;

/*
 * Undirected weighted graph as a symmetric CSR (the paper's G(V,E,W), Sec. 2:
 * positive edge weights; undirected per Table 1).
 *   n          number of vertices, 1 <= n < 2^31
 *   num_arcs   row_ptr[n] = 2|E| (every edge stored in both directions)
 *   row_ptr    [n+1] uint64, row_ptr[0] = 0, non-decreasing
 *   col        [num_arcs] uint32 < n; each row strictly increasing (no
 *              duplicate arcs); self-loops are not allowed
 *   w          [num_arcs] uint32 >= 1; the arc v->u and the arc u->v carry
 *              the same weight
 *   mem        where row_ptr, col and w live
 * chl_build rejects (CHL_EINVAL) any violation, including an arc without its
 * reverse.
 */
typedef struct {
    uint32_t n;
    uint64_t num_arcs;
    const uint64_t *row_ptr;
    const uint32_t *col;
    const uint32_t *w;
    chl_mem mem;
} chl_csr;

/* Labels produced by chl_build: opaque, library-owned, resident in device
   memory until chl_labels_free. */
typedef struct chl_labels chl_labels;

/*
 * Build options. Zero-initialise and set what you need; 0 means "choose
 * automatically" (the autotuner).
 *   root_begin, root_end   build only trees whose root has rank position p in
 *                          [root_begin, root_end), p = n-1-R(root) (p = 0 is
 *                          the most important vertex). root_end = 0 means n.
 *                          Trees are independent (Sec. 5.2), so disjoint
 *                          ranges partition the labels by hub.
 *   threads_per_tree       CUDA threads cooperating on one tree (a power of
 *                          two in [32, 1024])
 *   bucket_delta           distance width of one bucket of the tree search
 *                          (>= 1)
 *   window_buckets         buckets held in the near window (2..64)
 *   slots                  trees in flight at once
 *   mode                   0 = persistent batched launch (all roots claimed
 *                          dynamically in rank order by one launch);
 *                          1 = plain: one launch per root (one CTA of
 *                          threads_per_tree threads, default 512, builds it)
 *   flags                  bit set of CHL_FLAG_*; other bits are rejected
 *   label_capacity         initial size of the label buffer in labels; when
 *                          a tree does not fit, the buffer doubles and the
 *                          roots that did not fit are built again
 *   common_hubs            eta of the Common Label Table (Sec. 5.3): the trees
 *                          of the eta most important roots are built first and
 *                          all their labels kept in a table; every other tree
 *                          skips (no label, no relaxation) a vertex whose
 *                          distance query on that table is at most its tree
 *                          distance. The labels are unchanged. 0 = the paper's
 *                          eta = 16; negative = no table; at most
 *                          CHL_MAX_COMMON_HUBS. Requested trees of the eta
 *                          most important roots are built unpruned.
 *   pruned_bucket_delta    bucket width of the hybrid phases that prune with
 *                          the labels of earlier phases (their trees are
 *                          small, so wide buckets save rounds); 0 = the power
 *                          of two nearest twice the mean arc weight
 *   psi_threshold          Psi_th of the hybrid switch (Sec. 5.2): once a
 *                          phase expands more than Psi_th vertices per label it
 *                          generates, the later phases prune with the labels of
 *                          the earlier ones. 0 = 16, and the switch also fires
 *                          once the Common Label Table pruned at least 10% of
 *                          a phase's expansions; a value set here uses Psi
 *                          alone (the paper's 16-node runs use 100 on
 *                          scale-free and 500 on road networks, where the
 *                          switch also costs communication). Not negative.
 *   pruned_threads_per_tree  CUDA threads per tree in the phases that prune
 *                          with the labels of earlier phases (a power of two
 *                          in [32, 1024]); smaller blocks put more of those
 *                          small trees in flight. 0 = threads_per_tree
 *   switch_ratio           first-phase switch of the hybrid: when the labels
 *                          of the first phase (one tree per slot), per arc of
 *                          the graph, stay below this ratio, the label-pruned
 *                          phases start right after it. Scale-free graphs give
 *                          about 1.4 (R-MAT) to 3 (Barabasi-Albert), grids
 *                          above 10, where label pruning costs more than it
 *                          saves. 0 = 6 (and only when psi_threshold is 0);
 *                          negative = never (the Psi rule alone decides)
 *   round_limit            expansion rounds one tree may take before the
 *                          build stops with CHL_ETIMEOUT (0 = 2^26, far above
 *                          any tree of a graph below 2^31 vertices; a small
 *                          value makes the bounded-wait path testable)
 *   query_stage_kb         KiB of shared memory per tree slot in which the
 *                          label-pruned phases stage the label lists their
 *                          distance queries read, copied by the copy engine
 *                          (cp.async.bulk) instead of register loads; 0 = off
 *                          (measured slower on the R-MAT and grid workloads,
 *                          kept for other graphs and hardware)
 *   small_tree_expansions  frontier-size switch of the label-pruned phases:
 *                          once a phase's trees averaged fewer expansions than
 *                          this, the later phases (whose trees are smaller
 *                          still) run small_threads_per_tree threads per tree,
 *                          so that more trees share each SM and hide each
 *                          other's per-tree latency. 0 = 8192
 *   small_threads_per_tree threads per tree after that switch (a power of two
 *                          in [32, 1024]); 0 = 256 (or pruned_threads_per_tree
 *                          when smaller)
 *   big_tree_bucket_delta  bucket width of a label-pruned phase whose previous
 *                          phase's trees averaged at least 45% of the vertices
 *                          (big trees: narrow buckets cut the re-expansions of
 *                          a label-correcting search by more than they add in
 *                          rounds); 0 = pruned_bucket_delta / 16 (at least 1),
 *                          negative = pruned_bucket_delta for every phase
 *   overlap_phases         0 = on: while a label-pruned phase's last trees run,
 *                          the SMs they leave idle start the next phase's
 *                          first trees on a second stream, pruned by the
 *                          current (older) table; the labels are the same.
 *                          Negative = off (each phase waits for the last)
 */
/* chl_build_opts.flags: use 8-byte tree keys even where 4-byte keys hold
   every distance (the library picks 4 bytes when w_max * n < 2^31 - 1; the
   labels are the same either way). */
#define CHL_FLAG_WIDE_KEYS 1
/* chl_build_opts.flags: store with every label (h, d) of v the parent of v in
   the shortest-path tree of h (the next vertex from v towards h; h itself for
   the label of h), which lets chl_path return shortest paths in time linear in
   their length (Sec. 5.4, Extensions). Keys become 8 bytes; labels take 16
   instead of 12 bytes. Among several shortest-path predecessors the one with
   the highest rank is stored, so the parents are unique for a fixed R. */
#define CHL_FLAG_PARENTS 2
/* chl_build_opts.flags: run a build that starts at the top root as a single
   phase (no hybrid pruning). By default such a build runs its roots in phases
   of doubling size, and the trees of each phase also skip a vertex whose
   distance query over all labels of the earlier phases is at most its
   distance (the PLaNT-to-label-pruning hybrid of Sec. 5.2, on one GPU: the
   earlier phases' hubs form a rank-closed set, so the labels stay canonical
   and no cleaning pass is needed). */
#define CHL_FLAG_NO_HYBRID 4
/* chl_build_opts.flags: in the phases that prune with the labels of earlier
   phases, keep every root's labels in a per-slot array indexed by hub (by
   default only roots with more than 512 such labels do; the others hash them
   in shared memory). The labels are the same either way. */
#define CHL_FLAG_DENSE_ROOT_LABELS 8

typedef struct {
    uint32_t root_begin;
    uint32_t root_end;
    int32_t threads_per_tree;
    int32_t bucket_delta;
    int32_t window_buckets;
    int32_t slots;
    int32_t mode;
    int32_t flags;
    uint64_t label_capacity;
    int32_t common_hubs;
    int32_t pruned_bucket_delta;
    float psi_threshold;
    int32_t pruned_threads_per_tree;
    float switch_ratio;
    uint32_t round_limit;
    int32_t query_stage_kb;
    uint32_t small_tree_expansions;
    int32_t small_threads_per_tree;
    int32_t big_tree_bucket_delta;
    int32_t overlap_phases;
} chl_build_opts;

#define CHL_MAX_COMMON_HUBS 64


/*
 * Counters of a finished build (for throughput and exploration reports).
 *   trees          trees built (roots in the requested range)
 *   labels         total labels (hub, dist) emitted
 *   expanded       vertex expansions, re-expansions included
 *   arcs           arcs relaxed
 *   trivial        trees that ended at the root (every neighbour outranks it)
 *   build_ms       device time of the whole chl_build (CUDA events)
 *   tree_ms        device time of the tree kernel alone
 *   sort_ms        device time of label assembly (count, scan, scatter, sort)
 *   launches       kernels launched by the build
 *   rounds         expansion rounds of the tree searches (all trees)
 *   buckets        distance buckets entered after the first (all trees)
 *   pruned         expansions cut by the Common Label Table or by the label
 *                  table of earlier phases (all trees)
 *   table_ms       device time of building the Common Label Table (part of
 *                  tree_ms): its trees and the fill, or in a hybrid build,
 *                  whose first phase holds the table's trees, the fill alone;
 *                  0 without a table
 *   phases         tree phases run (1 unless the build is hybrid)
 *   label_table_phases  phases whose trees pruned with the label table of the
 *                  earlier ones (0: the switch threshold was never passed)
 *   small_tree_phases  label-pruned phases run with the small-tree launch
 *                  (the switch on small_tree_expansions; 0: it never fired)
 *   overlapped_trees  trees built in an earlier phase's tail on the second
 *                  stream (overlap_phases; trivial roots included), all of
 *                  whose labels were kept
 */
typedef struct {
    uint64_t trees;
    uint64_t labels;
    uint64_t expanded;
    uint64_t arcs;
    uint64_t trivial;
    double build_ms;
    double tree_ms;
    double sort_ms;
    uint64_t launches;
    uint64_t rounds;
    uint64_t buckets;
    uint64_t pruned;
    double table_ms;
    uint64_t phases;
    uint64_t label_table_phases;
    uint64_t small_tree_phases;
    uint64_t overlapped_trees;
} chl_build_stats;

/*
 * chl_build — canonical hub labels of g under ranking `rank` (PLaNT,
 * Sec. 5.2, Algorithm 3; early termination as in Sec. 5.2; label sort as in
 * Algorithm 2).
 *   g        input graph (see chl_csr); g->mem says where its arrays are
 *   rank     [n] uint32 R(v), a permutation of [0,n); same memory kind as g
 *   opts     NULL = defaults
 *   stream   cudaStream_t to order the work on
 *   out      receives the new labels object (owned by the caller, free with
 *            chl_labels_free); *out is NULL on failure
 * Errors: CHL_EINVAL (malformed graph, rank not a permutation, bad options),
 * CHL_ENOMEM, CHL_ECUDA, CHL_EOVERFLOW (a shortest distance reaches
 * UINT32_MAX, or one vertex holds more labels than the sorter supports).
 * With CHL_TRACE=1 in the environment a build prints one line per phase to
 * stderr (roots, tree and table times, expansions, arcs, labels); the extra
 * stream synchronisation makes traced builds slightly slower.
 */
chl_status chl_build(const chl_csr *g, const uint32_t *rank, const chl_build_opts *opts,
                     void *stream, chl_labels **out);

/*
 * chl_tune — pick the search parameters of chl_build for a graph by
 * measurement (the paper has no counterpart; its parameters α, β and Ψ_th
 * belong to other algorithms). The tree kernel runs on a rank-strided sample
 * of about four roots per tree slot (every (n/K)-th rank position, so the
 * sample has the build's mix of large and small trees) for candidate bucket
 * widths, then block sizes, then window sizes (coordinate search), and the
 * fastest is kept. For a whole build (no root range set in base) the block
 * size is then settled by whole builds (256, 512 and 1024 threads), since the
 * hybrid phases prune later trees far below the sample's sizes, and then the
 * phases' switch points, each by whole builds: the first-phase switch
 * (switch_ratio default or off), the frontier size of the small-tree switch
 * (small_tree_expansions 2048, 8192 or 32768), the narrow bucket width
 * after big trees (big_tree_bucket_delta default or off) and, for a build with
 * label-pruned phases, the Common Label Table's size (common_hubs 16, 8 or 4).
 *   g, rank, stream   as for chl_build
 *   base              fields set (non-zero) are kept fixed; NULL = tune all
 *   best              receives base with threads_per_tree, bucket_delta and
 *                     window_buckets filled in (and, for a whole build,
 *                     switch_ratio, small_tree_expansions,
 *                     big_tree_bucket_delta and common_hubs when base left
 *                     them 0); pass it to chl_build
 *   report            optional: trials run, sample size, best trial time
 * Errors: as chl_build.
 */
typedef struct {
    int32_t trials;
    uint32_t sample_roots;
    double best_tree_ms;
    uint64_t best_expanded;
    uint64_t best_arcs;
} chl_tune_report;

chl_status chl_tune(const chl_csr *g, const uint32_t *rank, const chl_build_opts *base,
                    void *stream, chl_build_opts *best, chl_tune_report *report);

/* n, total number of labels (the labeling's size, sum of |L_v|: the paper's
   ALS times n, Sec. 7.1 and Table 3), and device bytes held by the object.
   Any output pointer may be NULL. Errors: CHL_EINVAL (L is NULL). */
chl_status chl_labels_info(const chl_labels *L, uint32_t *n, uint64_t *total, uint64_t *bytes);

/* Counters of the build that produced L (see chl_build_stats). */
chl_status chl_labels_stats(const chl_labels *L, chl_build_stats *stats);

/*
 * Device views, valid until chl_labels_free(L). The labels are stored once,
 * per vertex (as the paper stores them for its shared-memory runs, Sec. 7.2
 * footnote), each list in the order the sort step of Algorithm 2 gives it
 * (by hub rank):
 *   offsets  [n+1] uint64; the labels of vertex v are entries
 *            [offsets[v], offsets[v+1])
 *   hub      [total] uint32 hub vertex id; within each vertex sorted by
 *            R(hub) descending (most important first); the last entry of
 *            L_v is v itself with distance 0
 *   dist     [total] uint32 d(v, hub)
 * Any output pointer may be NULL. The pointers are device memory of the
 * device L was built on; the library keeps ownership. Errors: CHL_EINVAL (L is
 * NULL).
 */
chl_status chl_labels_view(const chl_labels *L, const uint64_t **offsets, const uint32_t **hub,
                           const uint32_t **dist);

/*
 * Copy the labels (the per-vertex, hub-rank-sorted lists of chl_labels_view:
 * Algorithm 2's sort step, Sec. 7.2 footnote) into caller buffers (offsets
 * [n+1], hub [total], dist [total]; any may be NULL) in memory of kind
 * dst_mem, ordered on stream; returns after the copy completed.
 * Errors: CHL_EINVAL (L is NULL, unknown memory kind, or the current device is
 * not the one L was built on), CHL_ECUDA.
 */
chl_status chl_labels_copy(const chl_labels *L, uint64_t *offsets, uint32_t *hub, uint32_t *dist,
                           chl_mem dst_mem, void *stream);

/*
 * chl_query — PPSD queries (Sec. 1 cover property; Sec. 6 QLSN merge).
 *   pairs    [q][2] uint32 vertex ids (u, v), device or host per `mem`
 *   q        number of pairs (0 is allowed and does nothing)
 *   out      [q] uint32, out[i] = d(u_i, v_i), UINT32_MAX if u_i and v_i are
 *            disconnected; same memory kind as pairs
 * Errors: CHL_EINVAL (NULL pointers, a vertex id >= n, or the current device
 * is not the one L was built on), CHL_ENOMEM, CHL_ECUDA.
 */
chl_status chl_query(const chl_labels *L, const uint32_t *pairs, uint64_t q, uint32_t *out,
                     chl_mem mem, void *stream);

/*
 * chl_query_noalloc — the same queries as chl_query, without allocating any
 * memory. The paper has no counterpart: this entry point exists for callers
 * that must not allocate device memory on the query path, such as a serving
 * thread running inside a memory budget owned by another runtime, or one that
 * cannot take the allocator's synchronisation.
 *   L, pairs, q, out, mem, stream   as for chl_query
 * Scratch: one fixed device array inside the library (about 12 MiB, held on
 * every GPU that loads the library until the process exits) stages the pairs
 * and answers of host-memory calls and holds the bad-vertex flag.
 * Limits and rules:
 *   - q <= 1048576 (2^20) pairs per call; larger q returns CHL_EINVAL.
 *   - The first call on a device resolves the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream capture.
 *   - Each call synchronises `stream` before it returns (it reads the
 *     bad-vertex flag back to the host).
 *   - Every call uses the same array: calls whose work overlaps on the GPU
 *     (other streams, other host threads) race and must be serialised by the
 *     caller.
 * Errors: as chl_query.
 */
chl_status chl_query_noalloc(const chl_labels *L, const uint32_t *pairs, uint64_t q, uint32_t *out,
                             chl_mem mem, void *stream);

/*
 * chl_query_partitioned — PPSD queries over labels held as hub partitions: the
 * paper's fully distributed query mode (QFDL, Sec. 6: every node holds the
 * labels of its own hubs; each computes the partial minimum of
 * d(u,h) + d(v,h) over its hubs h in L_u and L_v, and a min-reduction combines
 * them) on one GPU. parts[k] holds the labels whose hubs lie in one rank
 * range (chl_build with root_begin/root_end); trees are independent (Sec.
 * 5.2), so disjoint ranges covering [0, n) partition the labeling by hub and
 * the answer equals chl_query's on the whole labeling.
 *   parts, nparts  1 <= nparts <= CHL_MAX_PARTS labels objects over the same n
 *                  vertices, all on the current device (caller keeps them)
 *   pairs, q, out, mem, stream  as for chl_query
 * Each pair is answered by one warp that merges the pair's partial lists of
 * every part and keeps the minimum.
 * Errors: CHL_EINVAL (NULL, nparts out of range, parts of different n or on
 * another device, a vertex id >= n), CHL_ENOMEM, CHL_ECUDA.
 */
#define CHL_MAX_PARTS 64
chl_status chl_query_partitioned(const chl_labels *const *parts, uint32_t nparts, const uint32_t *pairs,
                                 uint64_t q, uint32_t *out, chl_mem mem, void *stream);

/*
 * chl_query_grouped — the same answers as chl_query, with the batch answered
 * in grouped order: the paper's distributed query mode with labels owned by
 * vertex (QDOL, Sec. 6) sorts a batch by the vertex partitions its pairs need
 * and rearranges the answers back; on one GPU the partitions are 64 blocks of
 * vertex ids, a pair's key is the block pair (min(u,v), max(u,v)), the batch is
 * counting-sorted by key on the GPU, answered in that order (pairs that read
 * the lists of the same two blocks run together) and every answer is written
 * to its pair's slot in arrival order.
 *   L, pairs, q, out, mem, stream  as for chl_query (q < 2^32)
 * Errors: as chl_query.
 */
chl_status chl_query_grouped(const chl_labels *L, const uint32_t *pairs, uint64_t q, uint32_t *out,
                             chl_mem mem, void *stream);

/*
 * Copy the SPT parent of every label (caller vertex ids, [T], aligned with the
 * hub/dist arrays of chl_labels_copy) to host or device memory (mem).
 * CHL_EINVAL when L was built without CHL_FLAG_PARENTS.
 */
chl_status chl_labels_parents(const chl_labels *L, uint32_t *parent, chl_mem mem, void *stream);

/*
 * Shortest paths for q pairs (uint32 [q][2] caller ids). For each pair the
 * canonical hub H (the highest-ranked hub among those with the minimum
 * d(u,H) + d(H,v), i.e. the highest-ranked vertex on its shortest paths) is
 * found by the query merge; the path then follows the stored parents from u
 * to H and from v to H (Sec. 5.4, Extensions): time linear in its length.
 *   paths  [q][max_len] vertex ids, u first and v last; entries past the
 *          path's length (or past max_len) are left untouched
 *   lens   [q] vertices on the path (1 for u = v, 0 when u and v are not
 *          connected); a value above max_len means the path was cut there
 *   mem    where pairs, paths and lens live
 * Errors: CHL_EINVAL (NULL, id >= n, labels without parents, or the current
 * device is not the one L was built on).
 */
chl_status chl_path(const chl_labels *L, const uint32_t *pairs, uint64_t q, uint32_t max_len,
                    uint32_t *paths, uint32_t *lens, chl_mem mem, void *stream);

/* Release the labels object and its device arrays (NULL is allowed); the
   counterpart of chl_build, which hands ownership to the caller. The arrays
   are freed on the device L was built on, whatever device is current; the
   call synchronises that device. */
void chl_labels_free(chl_labels *L);

/* Message describing the last failure on the calling thread ("" if none). */
const char *chl_last_error(void);

/* Library version string. */
const char *chl_version(void);

/* ====================================================================== serving
 * A request loop on one GPU (the paper has no counterpart: it answers queries
 * one at a time from resident labels, Sec. 6 QLSN). Label sets stay resident in
 * device memory; PPSD queries that arrive while others are on the GPU are
 * gathered into the next batch (continuous batching) of one launch that may mix
 * label sets, with up to `query_slots` batches in flight on their own streams;
 * build requests run on worker threads and streams beside the queries and are
 * admitted in arrival order once their estimated device memory fits.
 * Streams share the device's hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS,
 * 8 by default, read when the CUDA context is created): with fewer queues than
 * streams, a query batch can wait behind a build's persistent tree kernel that
 * landed in the same queue. Set CUDA_DEVICE_MAX_CONNECTIONS=32 in the
 * environment before the process first uses CUDA.
 */
typedef struct chl_server chl_server;

/*
 * Server options. Zero-initialise; 0 selects the default.
 *   query_slots        batches in flight at once (default 3; each has its own
 *                      stream and pinned staging)
 *   max_batch          pairs per batch (default 1048576); a request larger than
 *                      this is rejected
 *   batching           0 = continuous batching (default); 1 = plain: one launch
 *                      per request, each waited for before the next (the
 *                      baseline the batching is measured against)
 *   build_workers      builds that may run at once (default 2)
 *   build_slots        SMs that running builds may hold together: a build
 *                      whose request sets neither opts.slots nor
 *                      opts.threads_per_tree runs build_slots / build_workers
 *                      slots of 1024 threads (one per SM). Default SMs - 16,
 *                      so that query batches keep SMs while trees run.
 *   build_budget       bytes that running builds may hold by their estimate
 *                      (default: free device memory at creation minus 4 GiB)
 *   query_order        0 = pairs of a batch answered in arrival order
 *                      (default); 1 = grouped: a batch larger than 4096 pairs
 *                      is sorted on the GPU by the vertex blocks its pairs
 *                      read (as chl_query_grouped) before it is answered
 */
typedef struct {
    int32_t query_slots;
    uint64_t max_batch;
    int32_t batching;
    int32_t build_workers;
    int32_t build_slots;
    uint64_t build_budget;
    int32_t query_order;
} chl_server_opts;

/* Counters since creation: batches launched, pairs answered, largest batch,
   builds admitted and finished, and the peak sum of admitted build estimates. */
typedef struct {
    uint64_t batches;
    uint64_t pairs;
    uint64_t max_batch_seen;
    uint64_t builds_done;
    uint64_t builds_failed;
    uint64_t build_bytes_peak;
} chl_server_stats;

/* Start a server on the current device (threads and streams are created).
   Errors: CHL_EINVAL, CHL_ENOMEM, CHL_ECUDA. */
chl_status chl_server_create(const chl_server_opts *opts, chl_server **out);

/* Make a label set resident for queries; *set_id receives its id (0, 1, ...,
   at most 4096 sets). L stays owned by the caller and must outlive every query
   on it. Call before submitting queries on it. */
chl_status chl_server_add_set(chl_server *S, const chl_labels *L, uint32_t *set_id);

/* Make a label set held as hub partitions resident (as chl_query_partitioned:
   parts[k] are labels of disjoint hub ranges over the same n vertices); its
   queries are answered by the minimum over the parts. The parts stay owned by
   the caller and must outlive every query on the set. Errors: CHL_EINVAL (NULL,
   nparts outside [1, CHL_MAX_PARTS], parts of different n or on another
   device, too many sets), CHL_ECUDA. */
chl_status chl_server_add_partitioned_set(chl_server *S, const chl_labels *const *parts,
                                          uint32_t nparts, uint32_t *set_id);

/* Queue `count` pairs (host uint32 [count][2], caller vertex ids of the set)
   for answers into host `out[count]`; both arrays must stay valid until the
   ticket completes. Ids are checked here: CHL_EINVAL for an id >= n, an unknown
   set, or count > max_batch. */
chl_status chl_server_submit_query(chl_server *S, uint32_t set_id, const uint32_t *pairs,
                                   uint64_t count, uint32_t *out, uint64_t *ticket);

/* Queue a build (as chl_build; g, rank and their arrays must stay valid until
   the ticket completes). Admitted in arrival order when its estimate (graph,
   slot state, labels at 256 per vertex) fits the budget and free memory. */
chl_status chl_server_submit_build(chl_server *S, const chl_csr *g, const uint32_t *rank,
                                   const chl_build_opts *opts, uint64_t *ticket);

/* Wait for a ticket (timeout_s < 0: no limit; CHL_ETIMEOUT when it runs out,
   the ticket stays valid). On completion returns the request's status, its
   latency from submission in *latency_s (optional) and, for a build, the new
   labels in *built (optional; owned by the caller, else freed). A ticket can be
   waited for once. */
chl_status chl_server_wait(chl_server *S, uint64_t ticket, double timeout_s, chl_labels **built,
                           double *latency_s);

/*
 * Open-loop replay: request i (pairs[pair_off[i] .. pair_off[i+1]) of set
 * set_of[i]) arrives arrival_s[i] seconds after the call starts (non-decreasing
 * times). The batcher takes every request that has arrived when a batch slot
 * frees, exactly as for submitted requests; latency_s[i] = completion -
 * arrival, answers into out[pair_off[i] ..]. *wall_s receives the time from the
 * start to the last completion. Submitted requests and builds keep being served
 * during the replay. Host arrays.
 */
chl_status chl_server_replay(chl_server *S, uint64_t nreq, const double *arrival_s,
                             const uint32_t *set_of, const uint64_t *pair_off,
                             const uint32_t *pairs, uint32_t *out, double *latency_s, double *wall_s);

chl_status chl_server_stats_get(const chl_server *S, chl_server_stats *stats);

/* Finish every queued request, stop the threads and free the server (NULL is
   allowed). Label sets added stay owned by the caller. */
void chl_server_destroy(chl_server *S);

#ifdef __cplusplus
}
#endif

#endif /* CHL_H */
