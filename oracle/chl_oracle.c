/*
 * CPU oracle for canonical hub labeling (CHL) and point-to-point shortest
 * distance (PPSD) queries.
 *
 * TEST INFRASTRUCTURE ONLY. This is a plain, slow, sequential-per-tree
 * restatement of what the paper defines. Only the test suite, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the GPU library never
 * calls it and shares no code with it.
 *
 * Notation (paper, Sec. 1 and Table 1): G(V,E,W) undirected with positive
 * integer weights; R a ranking function (a permutation of [0,n), larger R =
 * more important); SP_{u,v} the vertices on all shortest u-v paths, endpoints
 * included; L_v the labels (h, d(v,h)) of v.
 *
 * Three independent ways to build the labeling are provided; the paper proves
 * each yields the CHL (Sec. 1 definition; Sec. 5.2 PLaNT; Sec. 4 sequential PLL):
 *
 *   ORC_CANONICAL  the definition (Sec. 1; Lemma 1, Sec. 4.1): (h, d(v,h)) is
 *                  in L_v iff h is the highest-ranked vertex of SP_{v,h}.
 *                  Per root h: full Dijkstra, then best[v] = max rank over
 *                  SP_{h,v} by one pass over the settle order, label iff
 *                  best[v] == R(h).
 *   ORC_PLANT      Algorithm 3 (PLaNTDijkstra) in the paper's order and
 *                  notation, with early termination (cnt). Reading used: a
 *                  popped vertex outranked by nA gets no label but is still
 *                  relaxed; the paper states PLaNT does not prune trees
 *                  (Sec. 1, Sec. 5.2) and its termination rule counts such
 *                  vertices as explored.
 *   ORC_PLL        Algorithm 1 (pruned Dijkstra with rank queries) run
 *                  sequentially over roots in descending rank; sequential
 *                  PLL outputs the CHL (Sec. 4, proof of Claim 1).
 *   ORC_PLANT_CLT  PLaNT with the Common Label Table of Sec. 5.3: first the
 *                  trees of the eta most important roots (Algorithm 3, no
 *                  pruning); their labels, for every vertex, form the table
 *                  HC. Every other tree is Algorithm 3 in which a popped v is
 *                  pruned (no label, no relaxation) when a distance query on
 *                  HC, min over the table's hubs c of d(h,c) + d(c,v), is at
 *                  most delta_v. Sec. 5.3 states the resulting labels are not
 *                  redundant because HC holds all labels of every hub ranked
 *                  above any hub it prunes with.
 *
 * After construction every L_v is sorted by hub rank (Algorithm 2, line
 * "sort labels in L_v using hub rank"), most important hub first.
 *
 * Distances: uint64 accumulators during search; labels store uint32 and
 * UINT32_MAX is reserved for "unreachable". A build whose finite distance
 * reaches UINT32_MAX reports overflow.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <stdatomic.h>

#define ORC_CANONICAL 0
#define ORC_PLANT 1
#define ORC_PLL 2
#define ORC_PLANT_CLT 3

#define INF64 UINT64_MAX

typedef struct {
    uint64_t *offsets;  /* [n+1] */
    uint32_t *hub;      /* [total] */
    uint32_t *dist;     /* [total] */
    uint64_t total;
    int overflow;
} orc_labels;

void orc_free(void *p) { free(p); }

void orc_labels_free(orc_labels *L) {
    if (!L) return;
    free(L->offsets); free(L->hub); free(L->dist);
    memset(L, 0, sizeof(*L));
}

/* ------------------------------------------------------------------ indexed binary heap
 * Min-heap on (dist, tie) with decrease-key ("update Q" in Algorithms 1 and 3).
 * tie is the vertex id, or a seeded hash of it when randomised tie-breaking
 * is requested (used to show the output does not depend on the pop order of
 * equal distances). */
typedef struct {
    uint32_t *heap;     /* vertex ids */
    uint32_t *where;    /* position + 1, 0 = not in heap */
    uint64_t *key;      /* points to dist array */
    uint64_t tie_seed;
    size_t size;
} iheap;

static inline uint64_t tie_of(const iheap *q, uint32_t v) {
    if (!q->tie_seed) return v;
    uint64_t z = (uint64_t)v + q->tie_seed * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline int hless(const iheap *q, uint32_t a, uint32_t b) {
    if (q->key[a] != q->key[b]) return q->key[a] < q->key[b];
    uint64_t ta = tie_of(q, a), tb = tie_of(q, b);
    if (ta != tb) return ta < tb;
    return a < b;
}

static void hup(iheap *q, size_t i) {
    uint32_t v = q->heap[i];
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (!hless(q, v, q->heap[p])) break;
        q->heap[i] = q->heap[p];
        q->where[q->heap[i]] = (uint32_t)i + 1;
        i = p;
    }
    q->heap[i] = v;
    q->where[v] = (uint32_t)i + 1;
}

static void hdown(iheap *q, size_t i) {
    uint32_t v = q->heap[i];
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, s = i;
        uint32_t sv = v;
        if (l < q->size && hless(q, q->heap[l], sv)) { s = l; sv = q->heap[l]; }
        if (r < q->size && hless(q, q->heap[r], sv)) { s = r; sv = q->heap[r]; }
        if (s == i) break;
        q->heap[i] = sv;
        q->where[sv] = (uint32_t)i + 1;
        i = s;
    }
    q->heap[i] = v;
    q->where[v] = (uint32_t)i + 1;
}

/* insert v, or move it up after its key decreased */
static void hpush_or_decrease(iheap *q, uint32_t v) {
    if (q->where[v]) { hup(q, q->where[v] - 1); return; }
    q->heap[q->size] = v;
    hup(q, q->size++);
}

static uint32_t hpop(iheap *q) {
    uint32_t top = q->heap[0];
    q->where[top] = 0;
    if (--q->size) {
        q->heap[0] = q->heap[q->size];
        hdown(q, 0);
    }
    return top;
}

/* ------------------------------------------------------------------ per-thread workspace */
typedef struct {
    uint32_t v, hub;
    uint32_t dist;
} triple;

typedef struct {
    triple *buf;
    size_t len, cap;
} tbuf;

static int tpush(tbuf *b, uint32_t v, uint32_t hub, uint32_t dist) {
    if (b->len == b->cap) {
        size_t nc = b->cap ? 2 * b->cap : 1024;
        triple *nb = (triple *)realloc(b->buf, nc * sizeof(triple));
        if (!nb) return -1;
        b->buf = nb; b->cap = nc;
    }
    b->buf[b->len].v = v; b->buf[b->len].hub = hub; b->buf[b->len].dist = dist;
    b->len++;
    return 0;
}

typedef struct {
    uint64_t *dist;     /* delta_v, INF64 = unreached */
    uint32_t *anc;      /* a[v] (Algorithm 3) / best rank holder (definition) */
    uint32_t *order;    /* settle order */
    uint32_t *touched;  /* vertices whose entries were modified */
    uint64_t *lr;       /* the root's table labels by hub vertex, INF64 = none (phased method) */
    uint8_t *done;
    size_t ntouched;
    iheap q;
    tbuf out;
    int err;
    int overflow;
} workspace;

static int ws_init(workspace *w, uint32_t n, uint64_t tie_seed) {
    memset(w, 0, sizeof(*w));
    w->dist = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    w->anc = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    w->order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    w->touched = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    w->lr = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    w->done = (uint8_t *)calloc(n, 1);
    w->q.heap = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    w->q.where = (uint32_t *)calloc(n, sizeof(uint32_t));
    if (!w->dist || !w->anc || !w->order || !w->touched || !w->lr || !w->done || !w->q.heap ||
        !w->q.where)
        return -1;
    for (uint32_t v = 0; v < n; ++v) { w->dist[v] = INF64; w->anc[v] = v; w->lr[v] = INF64; }
    w->q.key = w->dist;
    w->q.tie_seed = tie_seed;
    return 0;
}

static void ws_free(workspace *w) {
    free(w->dist); free(w->anc); free(w->order); free(w->touched); free(w->lr); free(w->done);
    free(w->q.heap); free(w->q.where); free(w->out.buf);
}

/* reset only the entries the previous tree modified (footnote in Sec. 4.1) */
static void ws_reset(workspace *w) {
    for (size_t i = 0; i < w->ntouched; ++i) {
        uint32_t v = w->touched[i];
        w->dist[v] = INF64; w->anc[v] = v; w->done[v] = 0; w->q.where[v] = 0;
    }
    w->ntouched = 0;
    w->q.size = 0;
}

static inline void ws_touch(workspace *w, uint32_t v) {
    if (w->dist[v] == INF64) w->touched[w->ntouched++] = v;
}

typedef struct {
    uint32_t n;
    const uint64_t *row_ptr;
    const uint32_t *col;
    const uint32_t *w;
    const uint32_t *rank;
    /* Common Label Table (Sec. 5.3), or NULL: hc[v * eta + i] = d(v, c_i) when
       (c_i, d) is a label of v, UINT32_MAX otherwise, c_i the vertex of rank
       n-1-i (i = 0 most important) */
    const uint32_t *hc;
    uint32_t eta;
    /* label table of earlier phases (orc_build_phased), or lt_off = NULL:
       every label (hub, dist) of the roots of rank position below lt_hubs,
       CSR by vertex */
    const uint64_t *lt_off;
    const uint32_t *lt_hub;
    const uint32_t *lt_dist;
    uint32_t lt_hubs;
} graph;

/* per root: vertices settled, arcs scanned, labels, and label entries read by
   its distance queries (Algorithm 1 and the phased method) */
typedef struct { uint64_t settled, arcs, labels, qentries; } root_stats;

static int emit(workspace *ws, uint32_t v, uint32_t h, uint64_t d) {
    if (d >= UINT32_MAX) { ws->overflow = 1; d = UINT32_MAX - 1; }
    if (tpush(&ws->out, v, h, (uint32_t)d)) { ws->err = 1; return -1; }
    return 0;
}

/* ------------------------------------------------------------------ definition (Sec. 1) */
static void tree_canonical(const graph *g, workspace *ws, uint32_t h, root_stats *st) {
    /* 1. Dijkstra from h over the whole graph: d[.] and the settle order */
    uint64_t *d = ws->dist;
    size_t nset = 0;
    uint64_t arcs = 0;
    ws_touch(ws, h);
    d[h] = 0;
    hpush_or_decrease(&ws->q, h);
    while (ws->q.size) {
        uint32_t v = hpop(&ws->q);
        ws->done[v] = 1;
        ws->order[nset++] = v;
        for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            uint32_t u = g->col[e];
            arcs++;
            if (ws->done[u]) continue;
            uint64_t nd = d[v] + g->w[e];
            if (nd < d[u]) {
                ws_touch(ws, u);
                d[u] = nd;
                hpush_or_decrease(&ws->q, u);
            }
        }
    }
    /* 2. best[v] = max(R(v), max{best[p] : p in N(v), d[p] + w(p,v) = d[v]}),
          best[h] = R(h); every tight predecessor p has d[p] < d[v] (w >= 1),
          so it precedes v in the settle order. best is stored as the vertex
          holding that rank, in ws->anc. */
    uint32_t *best = ws->anc;
    best[h] = h;
    for (size_t i = 1; i < nset; ++i) {
        uint32_t v = ws->order[i];
        uint32_t b = v;
        for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            uint32_t p = g->col[e];
            if (d[p] != INF64 && d[p] + g->w[e] == d[v] && g->rank[best[p]] > g->rank[b]) b = best[p];
        }
        best[v] = b;
    }
    /* 3. label (h, d[v]) in L_v iff the highest rank on SP_{h,v} is R(h) */
    uint64_t nl = 0;
    for (size_t i = 0; i < nset; ++i) {
        uint32_t v = ws->order[i];
        if (best[v] == h) { if (emit(ws, v, h, d[v])) return; nl++; }
    }
    if (st) { st->settled = nset; st->arcs = arcs; st->labels = nl; }
}

/* ------------------------------------------------------------------ Algorithm 3 (PLaNTDijkstra) */
static inline uint32_t argmax_rank(const graph *g, uint32_t x, uint32_t y) {
    return g->rank[x] >= g->rank[y] ? x : y;
}

/* distance query on the Common Label Table between h and v (Sec. 5.3) */
static uint64_t hc_query(const graph *g, uint32_t h, uint32_t v) {
    uint64_t best = INF64;
    const uint32_t *a = g->hc + (uint64_t)h * g->eta, *b = g->hc + (uint64_t)v * g->eta;
    for (uint32_t i = 0; i < g->eta; ++i)
        if (a[i] != UINT32_MAX && b[i] != UINT32_MAX && (uint64_t)a[i] + b[i] < best)
            best = (uint64_t)a[i] + b[i];
    return best;
}

/* distance query between the root (its table labels in ws->lr) and v over the
   label table of earlier phases: some hub c with d(h,c) + d(c,v) <= dv; *qe
   counts the entries read */
static int lt_query_prunes(const graph *g, const workspace *ws, uint32_t v, uint64_t dv,
                           uint64_t *qe) {
    for (uint64_t i = g->lt_off[v]; i < g->lt_off[v + 1]; ++i) {
        ++*qe;
        const uint64_t dh = ws->lr[g->lt_hub[i]];
        if (dh != INF64 && dh + g->lt_dist[i] <= dv) return 1;
    }
    return 0;
}

static void tree_plant(const graph *g, workspace *ws, uint32_t h, root_stats *st) {
    uint64_t *delta = ws->dist;
    uint32_t *a = ws->anc;          /* a[v] = v for untouched v (ws_reset invariant) */
    const uint32_t Rh = g->rank[h];
    uint64_t settled = 0, arcs = 0, nl = 0, qe = 0;
    /* pruning by the Common Label Table applies to trees of roots outside it */
    const int prune = g->hc && g->n - 1 - Rh >= g->eta;
    /* pruning by the labels of earlier phases (phased method): the root's own
       table labels go into lr for the queries */
    const int lt = g->lt_off && g->n - 1 - Rh >= g->lt_hubs;
    if (lt)
        for (uint64_t i = g->lt_off[h]; i < g->lt_off[h + 1]; ++i) ws->lr[g->lt_hub[i]] = g->lt_dist[i];
    /* start: delta_h = 0, a[h] = h, h queued, cnt = 1 */
    ws_touch(ws, h);
    delta[h] = 0;
    a[h] = h;
    hpush_or_decrease(&ws->q, h);
    int64_t cnt = 1;
    while (ws->q.size) {
        if (cnt == 0) break;                                   /* early termination */
        uint32_t v = hpop(&ws->q);                             /* pop (v, delta_v) */
        ws->done[v] = 1;
        settled++;
        uint32_t nA = argmax_rank(g, v, a[v]);                 /* nA = argmax_{x in {v,a[v]}} R(x) */
        if (a[v] == h) cnt--;
        if (prune && hc_query(g, h, v) <= delta[v]) continue;  /* Sec. 5.3: pruned */
        if (lt && lt_query_prunes(g, ws, v, delta[v], &qe)) continue;  /* pruned by earlier phases */
        if (g->rank[nA] <= Rh) {                               /* R[nA] > R[h]: no label */
            if (emit(ws, v, h, delta[v])) return;              /* L_v = L_v U {(h, delta_v)} */
            nl++;
        }
        /* relax every arc of v, labelled or not (reading: trees are not pruned) */
        for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {
            uint32_t u = g->col[e];
            arcs++;
            uint32_t pA = a[u];
            uint64_t nd = delta[v] + g->w[e];
            if (ws->done[u]) continue;  /* settled: nd > delta_u, neither branch applies */
            if (nd < delta[u]) {
                a[u] = argmax_rank(g, nA, u);
            } else if (nd == delta[u]) {
                a[u] = argmax_rank(g, nA, pA);
            }
            if (a[u] == h && pA != h) cnt++;
            else if (a[u] != h && pA == h) cnt--;
            if (nd < delta[u]) {
                ws_touch(ws, u);
                delta[u] = nd;
                hpush_or_decrease(&ws->q, u);
            }
        }
    }
    if (lt) {
        qe += g->lt_off[h + 1] - g->lt_off[h];  /* the root's own list, read once */
        for (uint64_t i = g->lt_off[h]; i < g->lt_off[h + 1]; ++i) ws->lr[g->lt_hub[i]] = INF64;
    }
    if (st) { st->settled = settled; st->arcs = arcs; st->labels = nl; st->qentries = qe; }
}

/* ------------------------------------------------------------------ Algorithm 1 (sequential PLL) */
/* Labels built so far, per vertex, as growable arrays (hub, dist). */
typedef struct { uint32_t *hub; uint32_t *dist; uint32_t len, cap; } vlist;

static int vpush(vlist *l, uint32_t hub, uint32_t dist) {
    if (l->len == l->cap) {
        uint32_t nc = l->cap ? 2 * l->cap : 4;
        uint32_t *nh = (uint32_t *)realloc(l->hub, nc * sizeof(uint32_t));
        if (!nh) return -1;
        l->hub = nh;
        uint32_t *nd = (uint32_t *)realloc(l->dist, nc * sizeof(uint32_t));
        if (!nd) return -1;
        l->dist = nd; l->cap = nc;
    }
    l->hub[l->len] = hub; l->dist[l->len] = dist; l->len++;
    return 0;
}

static int build_pll(const graph *g, const uint32_t *roots, uint64_t nroots, uint64_t tie_seed,
                     tbuf *out, root_stats *stats, int *overflow) {
    const uint32_t n = g->n;
    vlist *L = (vlist *)calloc(n, sizeof(vlist));
    uint64_t *LR = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));  /* hash(L_h): dense table */
    workspace ws;
    if (!L || !LR || ws_init(&ws, n, tie_seed)) { free(L); free(LR); return -1; }
    for (uint32_t v = 0; v < n; ++v) LR[v] = INF64;
    int rc = 0;
    for (uint64_t ri = 0; ri < nroots && !rc; ++ri) {
        const uint32_t h = roots[ri];
        const uint32_t Rh = g->rank[h];
        uint64_t settled = 0, arcs = 0, nl = 0, qe = L[h].len;
        /* the root's labels by hub (LR), for the distance queries */
        for (uint32_t i = 0; i < L[h].len; ++i) LR[L[h].hub[i]] = L[h].dist[i];
        uint64_t *delta = ws.dist;
        ws_touch(&ws, h);
        delta[h] = 0;
        hpush_or_decrease(&ws.q, h);                             /* queue the root */
        while (ws.q.size) {
            uint32_t v = hpop(&ws.q);                            /* the closest queued vertex */
            ws.done[v] = 1;
            settled++;
            if (g->rank[v] > Rh) continue;                       /* rank query: v outranks h */
            /* distance query DQ(v, h, delta_v) over L_v and LR */
            int dq = 0;
            for (uint32_t i = 0; i < L[v].len && !dq; ++i) {
                ++qe;
                uint64_t dh = LR[L[v].hub[i]];
                if (dh != INF64 && (uint64_t)L[v].dist[i] + dh <= delta[v]) dq = 1;
            }
            if (dq) continue;
            if (delta[v] >= UINT32_MAX) *overflow = 1;
            if (vpush(&L[v], h, (uint32_t)delta[v])) { rc = -1; break; }   /* label (h, delta_v) */
            nl++;
            for (uint64_t e = g->row_ptr[v]; e < g->row_ptr[v + 1]; ++e) {  /* relax the arcs of v */
                uint32_t u = g->col[e];
                arcs++;
                if (ws.done[u]) continue;
                uint64_t nd = delta[v] + g->w[e];
                if (nd < delta[u]) {
                    ws_touch(&ws, u);
                    delta[u] = nd;
                    hpush_or_decrease(&ws.q, u);
                }
            }
        }
        for (uint32_t i = 0; i < L[h].len; ++i) LR[L[h].hub[i]] = INF64;
        ws_reset(&ws);
        if (stats) {
            stats[ri].settled = settled; stats[ri].arcs = arcs; stats[ri].labels = nl;
            stats[ri].qentries = qe;
        }
    }
    for (uint32_t v = 0; v < n && !rc; ++v)
        for (uint32_t i = 0; i < L[v].len; ++i)
            if (tpush(out, v, L[v].hub[i], L[v].dist[i])) { rc = -1; break; }
    for (uint32_t v = 0; v < n; ++v) { free(L[v].hub); free(L[v].dist); }
    free(L); free(LR);
    ws_free(&ws);
    return rc;
}

/* ------------------------------------------------------------------ threaded driver */
typedef struct {
    const graph *g;
    int method;
    const uint32_t *roots;
    uint64_t nroots;
    _Atomic uint64_t next;   /* dynamic claim of the next root (Sec. 4.1) */
    root_stats *stats;
    uint64_t tie_seed;
} job;

typedef struct { job *j; workspace ws; int rc; } worker;

static void *run_worker(void *arg) {
    worker *wk = (worker *)arg;
    job *j = wk->j;
    for (;;) {
        uint64_t i = atomic_fetch_add(&j->next, 1);
        if (i >= j->nroots) break;
        root_stats *st = j->stats ? &j->stats[i] : NULL;
        if (j->method == ORC_CANONICAL) tree_canonical(j->g, &wk->ws, j->roots[i], st);
        else tree_plant(j->g, &wk->ws, j->roots[i], st);
        ws_reset(&wk->ws);
        if (wk->ws.err) { wk->rc = -1; break; }
    }
    return NULL;
}

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/* counting sort of triples by v, then each L_v by R(hub) descending */
static int assemble(const graph *g, tbuf *parts, int nparts, orc_labels *out) {
    const uint32_t n = g->n;
    uint64_t total = 0;
    for (int p = 0; p < nparts; ++p) total += parts[p].len;
    out->offsets = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    out->hub = (uint32_t *)malloc(total * sizeof(uint32_t) + 4);
    out->dist = (uint32_t *)malloc(total * sizeof(uint32_t) + 4);
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!out->offsets || !out->hub || !out->dist || !fill) { free(fill); return -1; }
    for (int p = 0; p < nparts; ++p)
        for (size_t i = 0; i < parts[p].len; ++i) out->offsets[parts[p].buf[i].v + 1]++;
    for (uint32_t v = 0; v < n; ++v) out->offsets[v + 1] += out->offsets[v];
    memcpy(fill, out->offsets, ((size_t)n + 1) * sizeof(uint64_t));
    for (int p = 0; p < nparts; ++p)
        for (size_t i = 0; i < parts[p].len; ++i) {
            const triple *t = &parts[p].buf[i];
            uint64_t k = fill[t->v]++;
            out->hub[k] = t->hub; out->dist[k] = t->dist;
        }
    free(fill);
    /* sort each L_v by hub rank, most important first: key (n-1-R(hub)) << 32 | dist,
       ascending, then map the rank position back to the hub vertex */
    uint32_t *vert_at = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t maxlen = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (out->offsets[v + 1] - out->offsets[v] > maxlen) maxlen = out->offsets[v + 1] - out->offsets[v];
    uint64_t *keys = (uint64_t *)malloc((maxlen + 1) * sizeof(uint64_t));
    if (!vert_at || !keys) { free(vert_at); free(keys); return -1; }
    for (uint32_t v = 0; v < n; ++v) vert_at[n - 1 - g->rank[v]] = v;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t lo = out->offsets[v], len = out->offsets[v + 1] - lo;
        for (uint64_t i = 0; i < len; ++i)
            keys[i] = ((uint64_t)(n - 1 - g->rank[out->hub[lo + i]]) << 32) | out->dist[lo + i];
        qsort(keys, len, sizeof(uint64_t), cmp_u64);
        for (uint64_t i = 0; i < len; ++i) {
            out->hub[lo + i] = vert_at[keys[i] >> 32];
            out->dist[lo + i] = (uint32_t)keys[i];
        }
    }
    free(vert_at); free(keys);
    out->total = total;
    return 0;
}

/* Trees of roots[0..nroots) on `threads` threads with dynamic root claiming;
   each thread's (v, h, d) triples are returned in parts[threads]. */
static int run_trees(const graph *g, int method, const uint32_t *roots, uint64_t nroots, int threads,
                     uint64_t tie_seed, root_stats *stats, tbuf *parts, int *ovf) {
    int rc = 0;
    job j;
    j.g = g; j.method = method; j.roots = roots; j.nroots = nroots;
    atomic_init(&j.next, 0);
    j.stats = stats; j.tie_seed = tie_seed;
    worker *wk = (worker *)calloc((size_t)threads, sizeof(worker));
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!wk || !tid) { free(wk); free(tid); return -1; }
    for (int t = 0; t < threads; ++t) {
        wk[t].j = &j;
        if (ws_init(&wk[t].ws, g->n, tie_seed)) rc = -1;
    }
    if (!rc) {
        for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, run_worker, &wk[t]);
        run_worker(&wk[0]);
        for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    }
    for (int t = 0; t < threads; ++t) {
        if (wk[t].rc) rc = -1;
        *ovf |= wk[t].ws.overflow;
        parts[t] = wk[t].ws.out;
        wk[t].ws.out.buf = NULL;
        ws_free(&wk[t].ws);
    }
    free(wk); free(tid);
    return rc;
}

/*
 * Build labels with hubs in roots[0..nroots) (all vertices for a full build).
 * threads >= 1 (PLL always runs on one thread, in the given root order, which
 * must be descending rank for Algorithm 1). stats (optional) is indexed like
 * roots. eta: size of the Common Label Table for ORC_PLANT_CLT (1..n), else
 * ignored. Returns 0, -1 on allocation failure, -3 on bad arguments.
 */
int orc_build(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
              const uint32_t *rank, int method, const uint32_t *roots, uint64_t nroots,
              int threads, uint64_t tie_seed, uint32_t eta, orc_labels *out, root_stats *stats) {
    memset(out, 0, sizeof(*out));
    if (n == 0 || method < 0 || method > 3) return -3;
    if (method == ORC_PLANT_CLT && (eta < 1 || eta > n)) return -3;
    graph g = { n, row_ptr, col, w, rank, NULL, 0 };
    uint32_t *own_roots = NULL;
    if (!roots) {
        /* all vertices in descending rank (the paper's task queue order) */
        own_roots = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
        if (!own_roots) return -1;
        for (uint32_t v = 0; v < n; ++v) own_roots[n - 1 - rank[v]] = v;
        roots = own_roots;
        nroots = n;
    }
    if (threads < 1) threads = 1;
    int rc = 0, ovf = 0;
    if (method == ORC_PLL) {
        tbuf part = { 0 };
        rc = build_pll(&g, roots, nroots, tie_seed, &part, stats, &ovf);
        if (!rc) rc = assemble(&g, &part, 1, out);
        free(part.buf);
    } else if (method != ORC_PLANT_CLT) {
        tbuf *parts = (tbuf *)calloc((size_t)threads, sizeof(tbuf));
        if (!parts) { free(own_roots); return -1; }
        rc = run_trees(&g, method, roots, nroots, threads, tie_seed, stats, parts, &ovf);
        if (!rc) rc = assemble(&g, parts, threads, out);
        for (int t = 0; t < threads; ++t) free(parts[t].buf);
        free(parts);
    } else {
        /* 1. trees of the eta most important vertices, unpruned (Algorithm 3) */
        uint32_t *top = (uint32_t *)malloc((size_t)eta * sizeof(uint32_t));
        root_stats *tst = (root_stats *)calloc((size_t)eta, sizeof(root_stats));
        uint32_t *hc = (uint32_t *)malloc((size_t)n * eta * sizeof(uint32_t));
        tbuf *p1 = (tbuf *)calloc((size_t)threads, sizeof(tbuf));
        tbuf *p2 = (tbuf *)calloc((size_t)threads + 1, sizeof(tbuf));
        uint32_t *rest = (uint32_t *)malloc((size_t)nroots * sizeof(uint32_t) + 4);
        uint64_t *rest_at = (uint64_t *)malloc((size_t)nroots * sizeof(uint64_t) + 8);
        root_stats *rst = stats ? (root_stats *)calloc((size_t)nroots + 1, sizeof(root_stats)) : NULL;
        if (!top || !tst || !hc || !p1 || !p2 || !rest || !rest_at || (stats && !rst)) rc = -1;
        if (!rc) {
            for (uint32_t v = 0; v < n; ++v)
                if (n - 1 - rank[v] < eta) top[n - 1 - rank[v]] = v;
            rc = run_trees(&g, ORC_PLANT, top, eta, threads, tie_seed, tst, p1, &ovf);
        }
        if (!rc) {
            /* 2. the Common Label Table: every label of those eta hubs */
            for (size_t i = 0; i < (size_t)n * eta; ++i) hc[i] = UINT32_MAX;
            for (int t = 0; t < threads; ++t)
                for (size_t i = 0; i < p1[t].len; ++i) {
                    const triple *x = &p1[t].buf[i];
                    hc[(uint64_t)x->v * eta + (n - 1 - rank[x->hub])] = x->dist;
                }
            /* 3. every other requested tree, pruned by distance queries on HC */
            uint64_t nrest = 0;
            for (uint64_t i = 0; i < nroots; ++i)
                if (n - 1 - rank[roots[i]] >= eta) { rest_at[nrest] = i; rest[nrest++] = roots[i]; }
            g.hc = hc; g.eta = eta;
            rc = run_trees(&g, ORC_PLANT, rest, nrest, threads, tie_seed, rst, p2, &ovf);
            if (!rc && stats) {
                for (uint64_t k = 0; k < nrest; ++k) stats[rest_at[k]] = rst[k];
                for (uint64_t i = 0; i < nroots; ++i)
                    if (n - 1 - rank[roots[i]] < eta) stats[i] = tst[n - 1 - rank[roots[i]]];
            }
        }
        if (!rc) {
            /* requested labels: phase-3 trees plus the requested trees of phase 1 */
            uint8_t *want = (uint8_t *)calloc(eta, 1);
            if (!want) rc = -1;
            for (uint64_t i = 0; !rc && i < nroots; ++i)
                if (n - 1 - rank[roots[i]] < eta) want[n - 1 - rank[roots[i]]] = 1;
            for (int t = 0; !rc && t < threads; ++t)
                for (size_t i = 0; i < p1[t].len; ++i) {
                    const triple *x = &p1[t].buf[i];
                    if (want[n - 1 - rank[x->hub]] && tpush(&p2[threads], x->v, x->hub, x->dist)) rc = -1;
                }
            free(want);
            if (!rc) rc = assemble(&g, p2, threads + 1, out);
        }
        if (p1) for (int t = 0; t < threads; ++t) free(p1[t].buf);
        if (p2) for (int t = 0; t <= threads; ++t) free(p2[t].buf);
        free(top); free(tst); free(hc); free(p1); free(p2); free(rest); free(rest_at); free(rst);
    }
    out->overflow = ovf;
    free(own_roots);
    if (rc) orc_labels_free(out);
    return rc;
}

/*
 * Labels built in phases: the Hybrid of Sec. 5.2 in the form the library runs
 * it (reading R15 of the design notes: label-pruned phases instead of GLL
 * supersteps and cleaning). Phase k holds the roots of rank positions
 * [ends[k-1], ends[k]) (ends[-1] = 0, ends[nphases-1] <= n). With a last end
 * below n only the roots of rank positions below it are built: trees are
 * independent (Sec. 5.2), so those are the canonical labels whose hub ranks
 * among the top ends[nphases-1]. Its trees run
 * Algorithm 3 and also skip a popped vertex (no label, no relaxation) whose
 * distance query over every label of the earlier phases' roots is at most
 * its distance. Those roots are all hubs ranked above the phase's roots, the
 * condition Sec. 5.3 states for pruning without redundant labels, so the
 * result is the canonical labeling whatever the phases.
 * stats (optional, [n] by rank position). Returns as orc_build.
 */
int orc_build_phased(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, const uint32_t *w,
                     const uint32_t *rank, const uint32_t *ends, uint32_t nphases, int threads,
                     orc_labels *out, root_stats *stats) {
    memset(out, 0, sizeof(*out));
    if (n == 0 || nphases == 0 || ends[nphases - 1] > n) return -3;
    for (uint32_t k = 0; k < nphases; ++k)
        if (ends[k] == 0 || (k && ends[k] <= ends[k - 1])) return -3;
    if (threads < 1) threads = 1;
    graph g = { n, row_ptr, col, w, rank, NULL, 0 };
    uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *off = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *fill = (uint64_t *)calloc((size_t)n, sizeof(uint64_t));
    tbuf *parts = (tbuf *)calloc((size_t)threads, sizeof(tbuf));
    tbuf all = { 0 };
    uint32_t *thub = NULL, *tdist = NULL;
    int rc = 0, ovf = 0;
    if (!order || !off || !fill || !parts) rc = -1;
    if (!rc)
        for (uint32_t v = 0; v < n; ++v) order[n - 1 - rank[v]] = v;
    for (uint32_t k = 0; k < nphases && !rc; ++k) {
        const uint32_t pb = k ? ends[k - 1] : 0, pe = ends[k];
        if (k) {
            /* every label so far, as CSR by vertex */
            free(thub); free(tdist);
            thub = (uint32_t *)malloc(all.len * sizeof(uint32_t) + 4);
            tdist = (uint32_t *)malloc(all.len * sizeof(uint32_t) + 4);
            if (!thub || !tdist) { rc = -1; break; }
            memset(off, 0, ((size_t)n + 1) * sizeof(uint64_t));
            for (size_t i = 0; i < all.len; ++i) off[all.buf[i].v + 1]++;
            for (uint32_t v = 0; v < n; ++v) { off[v + 1] += off[v]; fill[v] = off[v]; }
            for (size_t i = 0; i < all.len; ++i) {
                const uint64_t at = fill[all.buf[i].v]++;
                thub[at] = all.buf[i].hub;
                tdist[at] = all.buf[i].dist;
            }
            g.lt_off = off; g.lt_hub = thub; g.lt_dist = tdist; g.lt_hubs = pb;
        }
        rc = run_trees(&g, ORC_PLANT, order + pb, pe - pb, threads, 0, stats ? stats + pb : NULL,
                       parts, &ovf);
        for (int t = 0; t < threads; ++t) {
            for (size_t i = 0; i < parts[t].len && !rc; ++i)
                if (tpush(&all, parts[t].buf[i].v, parts[t].buf[i].hub, parts[t].buf[i].dist)) rc = -1;
            free(parts[t].buf);
            memset(&parts[t], 0, sizeof(tbuf));
        }
    }
    if (!rc) rc = assemble(&g, &all, 1, out);
    out->overflow = ovf;
    free(parts); free(all.buf); free(order); free(off); free(fill); free(thub); free(tdist);
    if (rc) orc_labels_free(out);
    return rc;
}

/* ------------------------------------------------------------------ queries (Sec. 6, QLSN) */
/*
 * d(u,v) = min over common hubs h of d(u,h) + d(v,h) (Sec. 1): linear merge
 * of the two rank-sorted lists, scanned to the end. UINT32_MAX when no hub is
 * shared (disconnected pair); sums in uint64, saturated at UINT32_MAX.
 */
static uint32_t query_one(const uint64_t *off, const uint32_t *hub, const uint32_t *dist,
                          const uint32_t *rank, uint32_t u, uint32_t v) {
    uint64_t i = off[u], ie = off[u + 1], j = off[v], je = off[v + 1];
    uint64_t best = UINT32_MAX;
    while (i < ie && j < je) {
        uint32_t ru = rank[hub[i]], rv = rank[hub[j]];
        if (ru == rv) {
            uint64_t s = (uint64_t)dist[i] + dist[j];
            if (s < best) best = s;
            ++i; ++j;
        } else if (ru > rv) {
            ++i;
        } else {
            ++j;
        }
    }
    return (uint32_t)best;
}

typedef struct {
    const uint64_t *off; const uint32_t *hub; const uint32_t *dist; const uint32_t *rank;
    const uint32_t *pairs; uint64_t q; uint32_t *out; _Atomic uint64_t next;
} qjob;

static void *run_queries(void *arg) {
    qjob *j = (qjob *)arg;
    for (;;) {
        uint64_t b = atomic_fetch_add(&j->next, 4096);
        if (b >= j->q) break;
        uint64_t e = b + 4096 < j->q ? b + 4096 : j->q;
        for (uint64_t i = b; i < e; ++i)
            j->out[i] = query_one(j->off, j->hub, j->dist, j->rank, j->pairs[2 * i], j->pairs[2 * i + 1]);
    }
    return NULL;
}

int orc_query(uint32_t n, const uint64_t *offsets, const uint32_t *hub, const uint32_t *dist,
              const uint32_t *rank, const uint32_t *pairs, uint64_t q, uint32_t *out, int threads) {
    for (uint64_t i = 0; i < 2 * q; ++i)
        if (pairs[i] >= n) return -3;
    qjob j = { offsets, hub, dist, rank, pairs, q, out, 0 };
    atomic_init(&j.next, 0);
    if (threads < 1) threads = 1;
    pthread_t *tid = (pthread_t *)calloc((size_t)threads, sizeof(pthread_t));
    if (!tid) return -1;
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, run_queries, &j);
    run_queries(&j);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    free(tid);
    return 0;
}

/* ------------------------------------------------------------------ DQ_Clean (Algorithm 2) */
/*
 * Counts labels (h, delta) in L_v for which DQ_Clean returns true: the set W
 * of common hubs w of L_h and L_v with d(w,v) + d(w,h) <= delta holds a vertex
 * ranked above h. By Lemma 2 a labeling that respects R has no redundant label
 * iff this count is zero.
 */
uint64_t orc_count_redundant(uint32_t n, const uint64_t *off, const uint32_t *hub,
                             const uint32_t *dist, const uint32_t *rank) {
    uint64_t red = 0;
    for (uint32_t v = 0; v < n; ++v) {
        for (uint64_t k = off[v]; k < off[v + 1]; ++k) {
            const uint32_t h = hub[k];
            const uint64_t delta = dist[k];
            uint32_t best_rank = 0;
            int found = 0;
            uint64_t i = off[h], ie = off[h + 1], j = off[v], je = off[v + 1];
            while (i < ie && j < je) {
                uint32_t ri = rank[hub[i]], rj = rank[hub[j]];
                if (ri == rj) {
                    if ((uint64_t)dist[i] + dist[j] <= delta) {
                        if (!found || ri > best_rank) best_rank = ri;
                        found = 1;
                    }
                    ++i; ++j;
                } else if (ri > rj) ++i; else ++j;
            }
            if (found && best_rank > rank[h]) red++;
        }
    }
    return red;
}
