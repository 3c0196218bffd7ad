/*
 * Seeded synthetic inputs for canonical hub labeling: graphs (Barabasi-Albert,
 * R-MAT, 2-D grid), ranking functions R and query pairs.
 *
 * This file holds input synthesis only. It computes nothing of the labeling
 * method itself; both the CPU oracle and the GPU path consume what it writes.
 *
 * Random numbers: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014) seeds
 * xoshiro256** (Blackman, Vigna, 2018); bounded integers use Lemire's
 * multiply-and-reject method (ACM TOMACS 2019). Each (seed, stream) pair gives
 * an independent sequence, so graph structure, weights and queries do not
 * share draws.
 *
 * Output graphs are undirected, connected (largest component kept and
 * relabelled in id order), free of self-loops and duplicate edges, and stored
 * as a symmetric CSR: row_ptr[n+1] (uint64), col[2m] (uint32, each row sorted
 * by neighbour id), w[2m] (uint32, >= 1, equal on both arcs of an edge).
 *
 * Ranks follow the paper's convention (Sec. 1): R is a permutation of [0,n),
 * a larger R is a more important vertex. Degree ranking (Sec. 7.1, scale-free
 * graphs) sorts by degree descending, then id ascending; the road-like ranking
 * (Sec. 7.1 approximates betweenness by sampling shortest-path trees) counts,
 * for each vertex, the tree paths through it over seeded sample roots.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ------------------------------------------------------------------ RNG */
typedef struct { uint64_t s[4]; } gen_rng;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_init(gen_rng *r, uint64_t seed, uint64_t stream) {
    uint64_t sm = seed ^ (stream * 0xD1B54A32D192ED03ULL);
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&sm);
}

static uint64_t rng_next(gen_rng *r) {
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform integer in [0, range), range >= 1 */
static uint64_t rng_below(gen_rng *r, uint64_t range) {
    uint64_t x = rng_next(r);
    unsigned __int128 m = (unsigned __int128)x * range;
    uint64_t lo = (uint64_t)m;
    if (lo < range) {
        const uint64_t thresh = (0 - range) % range;
        while (lo < thresh) {
            x = rng_next(r);
            m = (unsigned __int128)x * range;
            lo = (uint64_t)m;
        }
    }
    return (uint64_t)(m >> 64);
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unit(gen_rng *r) { return (double)(rng_next(r) >> 11) * 0x1.0p-53; }

/* stream ids: one per purpose, so that changing one draw count never shifts another */
enum { ST_STRUCT = 1, ST_WEIGHT = 2, ST_DELETE = 3, ST_ROOTS = 4, ST_PAIRS = 5 };

/* ------------------------------------------------------------------ result */
typedef struct {
    uint32_t n;            /* vertices after largest-component extraction */
    uint64_t m;            /* undirected edges */
    uint64_t *row_ptr;     /* [n+1] */
    uint32_t *col;         /* [2m] */
    uint32_t *w;           /* [2m] */
    uint32_t n_before;     /* ids before extraction */
    uint64_t m_sampled;    /* edges drawn before clean-up */
} gen_graph;

void gen_free(void *p) { free(p); }

void gen_graph_free(gen_graph *g) {
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->w);
    g->row_ptr = NULL; g->col = NULL; g->w = NULL;
}

/* ------------------------------------------------------------------ sort */
/* LSD radix sort of 64-bit keys, 16 bits per pass */
static int radix_sort_u64(uint64_t *a, size_t n) {
    if (n < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc(n * sizeof(uint64_t));
    size_t *cnt = (size_t *)malloc(65536 * sizeof(size_t));
    if (!tmp || !cnt) { free(tmp); free(cnt); return -1; }
    uint64_t *src = a, *dst = tmp;
    for (int pass = 0; pass < 4; ++pass) {
        const int sh = 16 * pass;
        memset(cnt, 0, 65536 * sizeof(size_t));
        for (size_t i = 0; i < n; ++i) cnt[(src[i] >> sh) & 0xFFFF]++;
        size_t s = 0;
        for (size_t b = 0; b < 65536; ++b) { size_t c = cnt[b]; cnt[b] = s; s += c; }
        for (size_t i = 0; i < n; ++i) dst[cnt[(src[i] >> sh) & 0xFFFF]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    /* four passes: result is back in a */
    free(tmp); free(cnt);
    return 0;
}

/* ------------------------------------------------------------------ union-find */
static uint32_t uf_find(uint32_t *p, uint32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/*
 * keys: undirected edges as (lo << 32 | hi), lo < hi. Sorts, removes
 * duplicates, keeps the largest connected component (ties: the component
 * holding the smaller vertex id), relabels its vertices in id order, assigns
 * weights in sorted-edge order and writes the symmetric CSR.
 * weight_mode 0: uniform integer in [wlo, whi]; 1: llround(1000 * U[0.5,1.5)).
 */
static int finish_graph(uint64_t *keys, size_t nk, uint32_t nids, uint64_t seed,
                        int weight_mode, uint32_t wlo, uint32_t whi, gen_graph *out) {
    if (radix_sort_u64(keys, nk)) return -1;
    size_t m = 0;
    for (size_t i = 0; i < nk; ++i)
        if (m == 0 || keys[i] != keys[m - 1]) keys[m++] = keys[i];

    uint32_t *par = (uint32_t *)malloc((size_t)nids * sizeof(uint32_t));
    uint32_t *csize = (uint32_t *)calloc(nids, sizeof(uint32_t));
    uint8_t *touched = (uint8_t *)calloc(nids, 1);
    if (!par || !csize || !touched) { free(par); free(csize); free(touched); return -1; }
    for (uint32_t i = 0; i < nids; ++i) par[i] = i;
    for (size_t i = 0; i < m; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        touched[a] = touched[b] = 1;
        a = uf_find(par, a); b = uf_find(par, b);
        if (a != b) { if (a < b) par[b] = a; else par[a] = b; }  /* root = smallest id */
    }
    for (uint32_t i = 0; i < nids; ++i)
        if (touched[i]) csize[uf_find(par, i)]++;
    uint32_t best = 0, best_size = 0;
    for (uint32_t i = 0; i < nids; ++i)
        if (csize[i] > best_size) { best_size = csize[i]; best = i; }  /* first max = smallest id */
    uint32_t *newid = csize; /* reuse */
    uint32_t n = 0;
    for (uint32_t i = 0; i < nids; ++i)
        newid[i] = (touched[i] && uf_find(par, i) == best) ? n++ : UINT32_MAX;
    free(par); free(touched);
    if (n < 2) { free(newid); return -2; }

    size_t mm = 0;
    for (size_t i = 0; i < m; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        if (newid[a] == UINT32_MAX) continue;
        keys[mm++] = ((uint64_t)newid[a] << 32) | newid[b];  /* monotone relabel keeps order */
    }
    free(newid);

    uint64_t *row = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint32_t *col = (uint32_t *)malloc(2 * mm * sizeof(uint32_t) + 4);
    uint32_t *w = (uint32_t *)malloc(2 * mm * sizeof(uint32_t) + 4);
    uint32_t *ew = (uint32_t *)malloc(mm * sizeof(uint32_t) + 4);
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!row || !col || !w || !ew || !fill) {
        free(row); free(col); free(w); free(ew); free(fill); return -1;
    }
    gen_rng rw;
    rng_init(&rw, seed, ST_WEIGHT);
    for (size_t i = 0; i < mm; ++i) {
        if (weight_mode == 0) {
            ew[i] = wlo + (uint32_t)rng_below(&rw, (uint64_t)(whi - wlo) + 1);
        } else {
            double u = 0.5 + rng_unit(&rw);
            ew[i] = (uint32_t)llround(1000.0 * u);
        }
    }
    for (size_t i = 0; i < mm; ++i) {
        row[(keys[i] >> 32) + 1]++;
        row[(uint32_t)keys[i] + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) row[v + 1] += row[v];
    memcpy(fill, row, ((size_t)n + 1) * sizeof(uint64_t));
    /* lower neighbours first (edges (a,b), a<b, give b its neighbour a in increasing a) */
    for (size_t i = 0; i < mm; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        uint64_t p = fill[b]++;
        col[p] = a; w[p] = ew[i];
    }
    /* then upper neighbours, in increasing id */
    for (size_t i = 0; i < mm; ++i) {
        uint32_t a = (uint32_t)(keys[i] >> 32), b = (uint32_t)keys[i];
        uint64_t p = fill[a]++;
        col[p] = b; w[p] = ew[i];
    }
    free(ew); free(fill);
    out->n = n; out->m = mm; out->row_ptr = row; out->col = col; out->w = w;
    return 0;
}

/* ------------------------------------------------------------------ generators */

/*
 * Barabasi-Albert preferential attachment: a clique on m+1 vertices, then each
 * new vertex joins m distinct existing vertices drawn with probability
 * proportional to their degree (uniform draws from the list of edge endpoints).
 */
int gen_ba(uint32_t n, uint32_t m, uint64_t seed, uint32_t wlo, uint32_t whi, gen_graph *out) {
    memset(out, 0, sizeof(*out));
    if (m < 1 || n < m + 2) return -3;
    const size_t ne = (size_t)m * (m + 1) / 2 + (size_t)(n - m - 1) * m;
    uint64_t *keys = (uint64_t *)malloc(ne * sizeof(uint64_t));
    uint32_t *ends = (uint32_t *)malloc(2 * ne * sizeof(uint32_t));
    uint32_t *pick = (uint32_t *)malloc(m * sizeof(uint32_t));
    if (!keys || !ends || !pick) { free(keys); free(ends); free(pick); return -1; }
    size_t k = 0, ne2 = 0;
    for (uint32_t a = 0; a <= m; ++a)
        for (uint32_t b = a + 1; b <= m; ++b) {
            keys[k++] = ((uint64_t)a << 32) | b;
            ends[ne2++] = a; ends[ne2++] = b;
        }
    gen_rng r;
    rng_init(&r, seed, ST_STRUCT);
    for (uint32_t v = m + 1; v < n; ++v) {
        uint32_t got = 0;
        while (got < m) {
            uint32_t t = ends[rng_below(&r, ne2)];
            int dup = 0;
            for (uint32_t j = 0; j < got; ++j) dup |= (pick[j] == t);
            if (!dup) pick[got++] = t;
        }
        for (uint32_t j = 0; j < m; ++j) {
            keys[k++] = ((uint64_t)pick[j] << 32) | v;
            ends[ne2++] = pick[j]; ends[ne2++] = v;
        }
    }
    free(ends); free(pick);
    out->n_before = n; out->m_sampled = k;
    int rc = finish_graph(keys, k, n, seed, 0, wlo, whi, out);
    free(keys);
    return rc;
}

/*
 * R-MAT (Chakrabarti, Zhan, Faloutsos 2004): each edge descends `scale` levels
 * of the adjacency matrix, choosing quadrant (0,0),(0,1),(1,0),(1,1) with
 * probabilities a, b, c, 1-a-b-c; no noise, no id permutation. Then
 * symmetrised, self-loops and duplicates dropped, largest component kept.
 */
int gen_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c,
             uint64_t seed, uint32_t wlo, uint32_t whi, gen_graph *out) {
    memset(out, 0, sizeof(*out));
    if (scale < 2 || scale > 30) return -3;
    const uint32_t nids = 1u << scale;
    const size_t ne = (size_t)edge_factor << scale;
    uint64_t *keys = (uint64_t *)malloc(ne * sizeof(uint64_t));
    if (!keys) return -1;
    gen_rng r;
    rng_init(&r, seed, ST_STRUCT);
    const double ab = a + b, abc = a + b + c;
    size_t k = 0;
    for (size_t e = 0; e < ne; ++e) {
        uint32_t u = 0, v = 0;
        for (uint32_t lvl = 0; lvl < scale; ++lvl) {
            const double x = rng_unit(&r);
            uint32_t bu, bv;
            if (x < a) { bu = 0; bv = 0; }
            else if (x < ab) { bu = 0; bv = 1; }
            else if (x < abc) { bu = 1; bv = 0; }
            else { bu = 1; bv = 1; }
            u = (u << 1) | bu;
            v = (v << 1) | bv;
        }
        if (u == v) continue;
        keys[k++] = u < v ? (((uint64_t)u << 32) | v) : (((uint64_t)v << 32) | u);
    }
    out->n_before = nids; out->m_sampled = ne;
    int rc = finish_graph(keys, k, nids, seed, 0, wlo, whi, out);
    free(keys);
    return rc;
}

/*
 * side x side 4-neighbour grid (vertex id = row*side + col); exactly
 * `n_delete` edges removed uniformly without replacement (partial
 * Fisher-Yates over the edges in sorted order); largest component kept;
 * weights llround(1000 * U[0.5,1.5)).
 */
int gen_grid(uint32_t side, uint64_t n_delete, uint64_t seed, gen_graph *out) {
    memset(out, 0, sizeof(*out));
    if (side < 2) return -3;
    const uint32_t nids = side * side;
    const size_t ne = (size_t)2 * side * (side - 1);
    if (n_delete >= ne) return -3;
    uint64_t *keys = (uint64_t *)malloc(ne * sizeof(uint64_t));
    if (!keys) return -1;
    size_t k = 0;
    for (uint32_t rr = 0; rr < side; ++rr)
        for (uint32_t cc = 0; cc < side; ++cc) {
            uint32_t v = rr * side + cc;
            if (cc + 1 < side) keys[k++] = ((uint64_t)v << 32) | (v + 1);
            if (rr + 1 < side) keys[k++] = ((uint64_t)v << 32) | (v + side);
        }
    radix_sort_u64(keys, k);
    gen_rng r;
    rng_init(&r, seed, ST_DELETE);
    for (size_t i = 0; i < n_delete; ++i) {
        size_t j = i + (size_t)rng_below(&r, k - i);
        uint64_t t = keys[i]; keys[i] = keys[j]; keys[j] = t;
    }
    out->n_before = nids; out->m_sampled = ne;
    int rc = finish_graph(keys + n_delete, k - n_delete, nids, seed, 1, 0, 0, out);
    free(keys);
    return rc;
}

/* ------------------------------------------------------------------ ranks */

/* rank from a score: order by (score desc, id asc) gives pos; R = n-1-pos */
static int rank_from_score(uint32_t n, const uint64_t *score, uint32_t *rank_out) {
    /* one 64-bit key per vertex, (2^40-1-score) << 24 | id, sorted ascending:
       scores are clamped to 40 bits and ids must fit in 24 bits */
    uint64_t *k = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!k) return -1;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t s = score[v];
        if (s >= (1ULL << 40)) s = (1ULL << 40) - 1;
        k[v] = (((1ULL << 40) - 1 - s) << 24) | v;
    }
    if (n > (1u << 24)) { free(k); return -3; }
    radix_sort_u64(k, n);
    for (uint32_t p = 0; p < n; ++p) rank_out[k[p] & 0xFFFFFF] = n - 1 - p;
    free(k);
    return 0;
}

int gen_degree_rank(uint32_t n, const uint64_t *row_ptr, uint32_t *rank_out) {
    uint64_t *deg = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    if (!deg) return -1;
    for (uint32_t v = 0; v < n; ++v) deg[v] = row_ptr[v + 1] - row_ptr[v];
    int rc = rank_from_score(n, deg, rank_out);
    free(deg);
    return rc;
}

/* binary min-heap on (dist, vertex) used only by the sampled-tree ranking */
typedef struct { uint64_t d; uint32_t v; } hitem;
static void hpush(hitem *h, size_t *sz, uint64_t d, uint32_t v) {
    size_t i = (*sz)++;
    while (i > 0) {
        size_t p = (i - 1) / 2;
        if (h[p].d < d || (h[p].d == d && h[p].v <= v)) break;
        h[i] = h[p]; i = p;
    }
    h[i].d = d; h[i].v = v;
}
static hitem hpop(hitem *h, size_t *sz) {
    hitem top = h[0], last = h[--(*sz)];
    size_t i = 0;
    for (;;) {
        size_t l = 2 * i + 1, r = l + 1, s = i;
        hitem best = last;
        if (l < *sz && (h[l].d < best.d || (h[l].d == best.d && h[l].v < best.v))) { s = l; best = h[l]; }
        if (r < *sz && (h[r].d < best.d || (h[r].d == best.d && h[r].v < best.v))) { s = r; best = h[r]; }
        if (s == i) break;
        h[i] = h[s]; i = s;
    }
    if (*sz > 0) h[i] = last;
    return top;
}

/*
 * Betweenness-style ranking: for each of `samples` distinct seeded roots,
 * a shortest-path tree whose parent is the tight predecessor of smallest id;
 * score(v) += size of v's subtree (the number of tree paths through v).
 * Rank by score desc, id asc.
 */
int gen_spt_count_rank(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                       const uint32_t *w, uint32_t samples, uint64_t seed, uint32_t *rank_out) {
    if (samples > n) samples = n;
    uint64_t *score = (uint64_t *)calloc(n, sizeof(uint64_t));
    uint64_t *dist = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint32_t *parent = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *order = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *sub = (uint64_t *)malloc((size_t)n * sizeof(uint64_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint8_t *done = (uint8_t *)malloc(n);
    hitem *heap = (hitem *)malloc((row_ptr[n] + 1) * sizeof(hitem));
    int rc = -1;
    if (!score || !dist || !parent || !order || !sub || !perm || !done || !heap) goto out;
    gen_rng r;
    rng_init(&r, seed, ST_ROOTS);
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = 0; i < samples; ++i) {
        uint32_t j = i + (uint32_t)rng_below(&r, n - i);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (uint32_t s = 0; s < samples; ++s) {
        const uint32_t src = perm[s];
        for (uint32_t v = 0; v < n; ++v) { dist[v] = UINT64_MAX; parent[v] = UINT32_MAX; done[v] = 0; }
        size_t hs = 0, no = 0;
        dist[src] = 0;
        hpush(heap, &hs, 0, src);
        while (hs) {
            hitem it = hpop(heap, &hs);
            if (done[it.v]) continue;
            done[it.v] = 1;
            order[no++] = it.v;
            for (uint64_t e = row_ptr[it.v]; e < row_ptr[it.v + 1]; ++e) {
                const uint32_t u = col[e];
                const uint64_t nd = it.d + w[e];
                if (nd < dist[u]) { dist[u] = nd; hpush(heap, &hs, nd, u); }
            }
        }
        /* parent = tight predecessor of smallest id */
        for (size_t i = 1; i < no; ++i) {
            const uint32_t v = order[i];
            for (uint64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
                const uint32_t p = col[e];
                if (dist[p] != UINT64_MAX && dist[p] + w[e] == dist[v]) {
                    if (p < parent[v]) parent[v] = p;
                }
            }
        }
        for (size_t i = 0; i < no; ++i) sub[order[i]] = 1;
        for (size_t i = no; i-- > 1;) {
            const uint32_t v = order[i];
            sub[parent[v]] += sub[v];
        }
        for (size_t i = 0; i < no; ++i) score[order[i]] += sub[order[i]];
    }
    rc = rank_from_score(n, score, rank_out);
out:
    free(score); free(dist); free(parent); free(order); free(sub); free(perm); free(done); free(heap);
    return rc;
}

/* ------------------------------------------------------------------ queries */

/* q pairs (u, v), u and v i.i.d. uniform over [0, n) */
int gen_uniform_pairs(uint32_t n, uint64_t q, uint64_t seed, uint32_t *pairs) {
    gen_rng r;
    rng_init(&r, seed, ST_PAIRS);
    for (uint64_t i = 0; i < q; ++i) {
        pairs[2 * i] = (uint32_t)rng_below(&r, n);
        pairs[2 * i + 1] = (uint32_t)rng_below(&r, n);
    }
    return 0;
}

/* q pairs with both endpoints drawn with probability proportional to degree
   (the source of a uniformly drawn arc) */
int gen_degree_pairs(uint32_t n, const uint64_t *row_ptr, uint64_t q, uint64_t seed, uint32_t *pairs) {
    const uint64_t arcs = row_ptr[n];
    if (arcs == 0) return -3;
    gen_rng r;
    rng_init(&r, seed, ST_PAIRS + 16);
    for (uint64_t i = 0; i < 2 * q; ++i) {
        const uint64_t a = rng_below(&r, arcs);
        /* binary search the row holding arc a */
        uint32_t lo = 0, hi = n;
        while (hi - lo > 1) {
            uint32_t mid = lo + (hi - lo) / 2;
            if (row_ptr[mid] <= a) lo = mid; else hi = mid;
        }
        pairs[i] = lo;
    }
    return 0;
}

/* uniform doubles in [0,1) (e.g. arrival-time draws) */
int gen_unit_doubles(uint64_t count, uint64_t seed, uint64_t stream, double *out) {
    gen_rng r;
    rng_init(&r, seed, 64 + stream);
    for (uint64_t i = 0; i < count; ++i) out[i] = rng_unit(&r);
    return 0;
}
