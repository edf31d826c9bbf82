/*
 * CPU oracle for flow-based hypergraph refinement (Gottesbueren, Heuer,
 * Sanders, "Parallel Flow-Based Hypergraph Partitioning").
 *
 * TEST INFRASTRUCTURE ONLY.  Plain, slow and written to be checked by eye
 * against the paper.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may load this code; the CUDA library never
 * calls it and shares no code with it.
 *
 * Every routine works on the EXPLICIT Lawler expansion of the flow
 * hypergraph (Section 2, "Flows on Hypergraphs"): hypernodes, an in-node and
 * an out-node per net, infinite pin arcs (u, e_in) and (e_out, u), and a
 * bridge (e_in, e_out) of capacity w(e).  Lawler node numbering:
 *   hypernode h            -> h                  (0 = s, 1 = t, 2.. = region)
 *   in-node of net e       -> n_nodes + e
 *   out-node of net e      -> n_nodes + m_nets + e
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>

#define OR_OK 0
#define OR_ERR_INVALID (-1)
#define OR_ERR_OOM (-2)
#define OR_ITER_LIMIT (-4)
#define OR_NO_BALANCED_CUT (-5)
#define OR_ABORTED_WORSE (-6)
#define OR_ERR_BUFFER (-7)

#define DIST_FAR ((1 << 20) - 1)

/* ------------------------------------------------------------------------ */
/* Flow network construction: Section 6, "Construction Algorithms", the first
 * (net scan) algorithm.  For every net with a pin in the region B, region
 * pins are copied (in the net's pin order), and a pin outside B adds the
 * source s (its block is the S side, side 0) or the sink t (side 1), each at
 * most once per net.  Pins whose side is neither 0 nor 1 belong to neither
 * block of the pair and are dropped.  Nets with fewer than two pins left, or
 * holding both s and t, are discarded (Section 6, last paragraph of
 * "Construction Algorithms").  Kept nets keep ascending net id order.
 *
 * Returns the pin count of the flow hypergraph, or a negative error.
 * Output capacities: m nets, net_off[m] + 2m pins, n_region + 2 nodes.
 */
int64_t or_build_network(int32_t n, int32_t m, const uint32_t *net_off, const int32_t *pins,
                         const int32_t *net_w, const int32_t *node_w, const int32_t *side,
                         const int32_t *region, int32_t n_region,
                         int32_t *out_m, uint32_t *nnet_off, int32_t *npins, int32_t *nnet_w,
                         int32_t *nnet_gid, int64_t *nnode_w) {
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!loc) return OR_ERR_OOM;
    for (int32_t v = 0; v < n; v++) loc[v] = -1;
    for (int32_t i = 0; i < n_region; i++) {
        int32_t v = region[i];
        if (v < 0 || v >= n || loc[v] >= 0 || (side[v] != 0 && side[v] != 1)) {
            free(loc);
            return OR_ERR_INVALID;
        }
        loc[v] = 2 + i;
    }
    nnode_w[0] = 0;
    nnode_w[1] = 0;
    for (int32_t v = 0; v < n; v++) {
        int64_t c = node_w ? node_w[v] : 1;
        if (loc[v] >= 0) nnode_w[loc[v]] = c;
        else if (side[v] == 0) nnode_w[0] += c;
        else if (side[v] == 1) nnode_w[1] += c;
    }
    int64_t p = 0;
    int32_t mm = 0;
    for (int32_t e = 0; e < m; e++) {
        int64_t start = p;
        int has_s = 0, has_t = 0;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t v = pins[j];
            if (loc[v] >= 0) npins[p++] = loc[v];
            else if (side[v] == 0) has_s = 1;
            else if (side[v] == 1) has_t = 1;
        }
        int64_t cnt = (p - start) + has_s + has_t;
        if (cnt < 2 || (has_s && has_t)) { p = start; continue; }
        if (has_s) npins[p++] = 0;
        if (has_t) npins[p++] = 1;
        nnet_off[mm] = (uint32_t)start;
        nnet_w[mm] = net_w[e];
        nnet_gid[mm] = e;
        mm++;
    }
    nnet_off[mm] = (uint32_t)p;
    *out_m = mm;
    free(loc);
    return p;
}

/* ------------------------------------------------------------------------ */
/* Distance from the original cut (Section 6, "Region Growing", last
 * paragraph, and Section 7, "Piercing").  The paper does not define it; the
 * reading used here: hop distance inside the region B.  Region pins of a net
 * of H that has pins on both sides (side 0 and side 1) get distance 1; region
 * pins of a net containing a region vertex at distance d that are still
 * unlabelled get d + 1.  Unreached region vertices get DIST_FAR; values are
 * clamped to DIST_FAR.  dist is indexed by region position.
 */
int32_t or_dist_from_cut(int32_t n, int32_t m, const uint32_t *net_off, const int32_t *pins,
                         const int32_t *side, const int32_t *region, int32_t n_region,
                         int32_t *dist) {
    int32_t *loc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *deg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    if (!loc || !deg) { free(loc); free(deg); return OR_ERR_OOM; }
    for (int32_t v = 0; v < n; v++) loc[v] = -1;
    for (int32_t i = 0; i < n_region; i++) loc[region[i]] = i;
    /* vertex -> nets incidence of H, restricted to region vertices */
    for (int32_t e = 0; e < m; e++)
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++)
            if (loc[pins[j]] >= 0) deg[pins[j] + 1]++;
    for (int32_t v = 0; v < n; v++) deg[v + 1] += deg[v];
    int64_t tot = deg[n];
    int32_t *inc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(tot > 0 ? tot : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_region > 0 ? n_region : 1));
    if (!inc || !fill || !queue) { free(loc); free(deg); free(inc); free(fill); free(queue); return OR_ERR_OOM; }
    memcpy(fill, deg, sizeof(int32_t) * (size_t)n);
    for (int32_t e = 0; e < m; e++)
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++)
            if (loc[pins[j]] >= 0) inc[fill[pins[j]]++] = e;
    for (int32_t i = 0; i < n_region; i++) dist[i] = -1;
    int32_t qh = 0, qt = 0;
    for (int32_t e = 0; e < m; e++) {
        int s0 = 0, s1 = 0;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            if (side[pins[j]] == 0) s0 = 1;
            if (side[pins[j]] == 1) s1 = 1;
        }
        if (!(s0 && s1)) continue;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t i = loc[pins[j]];
            if (i >= 0 && dist[i] < 0) { dist[i] = 1; queue[qt++] = pins[j]; }
        }
    }
    while (qh < qt) {
        int32_t u = queue[qh++];
        int32_t du = dist[loc[u]];
        for (int32_t k = deg[u]; k < deg[u + 1]; k++) {
            int32_t e = inc[k];
            for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
                int32_t i = loc[pins[j]];
                if (i >= 0 && dist[i] < 0) {
                    dist[i] = du + 1 < DIST_FAR ? du + 1 : DIST_FAR;
                    queue[qt++] = pins[j];
                }
            }
        }
    }
    for (int32_t i = 0; i < n_region; i++) if (dist[i] < 0) dist[i] = DIST_FAR;
    free(loc); free(deg); free(inc); free(fill); free(queue);
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Explicit Lawler expansion (Section 2, "Flows on Hypergraphs"). */
typedef struct {
    int32_t n_nodes, m_nets, N;   /* hypernodes, nets, Lawler nodes */
    int64_t A;                    /* arcs, each edge stored with its reverse */
    int64_t *adj_off;             /* N + 1 */
    int32_t *head, *tail;
    int64_t *cap, *flow, *rev;
    int64_t inf;                  /* "infinite" capacity: 1 + sum of all w(e) */
    int64_t *node_w;              /* hypernode weights c(h) */
} Lawler;

void or_lawler_free(Lawler *G) {
    if (!G) return;
    free(G->adj_off); free(G->head); free(G->tail); free(G->cap); free(G->flow); free(G->rev);
    free(G->node_w);
    free(G);
}

Lawler *or_lawler_create(int32_t n_nodes, int32_t m_nets, const uint32_t *net_off,
                         const int32_t *npins, const int32_t *net_w, const int64_t *node_w) {
    Lawler *G = (Lawler *)calloc(1, sizeof(Lawler));
    if (!G) return NULL;
    G->n_nodes = n_nodes;
    G->m_nets = m_nets;
    G->N = n_nodes + 2 * m_nets;
    int64_t P = net_off[m_nets];
    int64_t E = 2 * P + m_nets;     /* edges: two per pin plus one bridge per net */
    G->A = 2 * E;
    G->adj_off = (int64_t *)calloc((size_t)G->N + 1, sizeof(int64_t));
    G->head = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G->A + 1));
    G->tail = (int32_t *)malloc(sizeof(int32_t) * (size_t)(G->A + 1));
    G->cap = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->A + 1));
    G->flow = (int64_t *)calloc((size_t)G->A + 1, sizeof(int64_t));
    G->rev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->A + 1));
    G->node_w = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n_nodes + 1));
    if (!G->adj_off || !G->head || !G->tail || !G->cap || !G->flow || !G->rev || !G->node_w) {
        or_lawler_free(G);
        return NULL;
    }
    memcpy(G->node_w, node_w, sizeof(int64_t) * (size_t)n_nodes);
    int64_t inf = 1;
    for (int32_t e = 0; e < m_nets; e++) inf += net_w[e];
    G->inf = inf;
    /* edge list */
    int32_t *eu = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
    int32_t *ev = (int32_t *)malloc(sizeof(int32_t) * (size_t)(E + 1));
    int64_t *ec = (int64_t *)malloc(sizeof(int64_t) * (size_t)(E + 1));
    if (!eu || !ev || !ec) { free(eu); free(ev); free(ec); or_lawler_free(G); return NULL; }
    int64_t k = 0;
    for (int32_t e = 0; e < m_nets; e++) {
        int32_t ein = n_nodes + e, eout = n_nodes + m_nets + e;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t u = npins[j];
            eu[k] = u; ev[k] = ein; ec[k] = inf; k++;      /* (u, e_in), infinite */
            eu[k] = eout; ev[k] = u; ec[k] = inf; k++;     /* (e_out, u), infinite */
        }
        eu[k] = ein; ev[k] = eout; ec[k] = net_w[e]; k++;  /* bridge, capacity w(e) */
    }
    for (int64_t i = 0; i < E; i++) { G->adj_off[eu[i] + 1]++; G->adj_off[ev[i] + 1]++; }
    for (int32_t x = 0; x < G->N; x++) G->adj_off[x + 1] += G->adj_off[x];
    int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)(G->N + 1));
    if (!pos) { free(eu); free(ev); free(ec); or_lawler_free(G); return NULL; }
    memcpy(pos, G->adj_off, sizeof(int64_t) * (size_t)G->N);
    for (int64_t i = 0; i < E; i++) {
        int64_t a = pos[eu[i]]++, b = pos[ev[i]]++;
        G->head[a] = ev[i]; G->tail[a] = eu[i]; G->cap[a] = ec[i]; G->rev[a] = b;
        G->head[b] = eu[i]; G->tail[b] = ev[i]; G->cap[b] = 0; G->rev[b] = a;
    }
    free(pos); free(eu); free(ev); free(ec);
    return G;
}

int32_t or_lawler_nodes(const Lawler *G) { return G->N; }
int64_t or_lawler_arcs(const Lawler *G) { return G->A; }

static int64_t residual(const Lawler *G, int64_t a) { return G->cap[a] - G->flow[a]; }

static void push_arc(Lawler *G, int64_t a, int64_t d) {
    G->flow[a] += d;
    G->flow[G->rev[a]] -= d;
}

/* Dinic's algorithm from the source set S to the sink set T, starting from
 * the flow already on the arcs (an S-T flow stays feasible when S or T grow,
 * so FlowCutter's "augment flow to maximality" continues from it).
 * Returns the amount of flow added. */
static int64_t dinic(Lawler *G, const uint8_t *src, const uint8_t *snk) {
    int32_t N = G->N;
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int64_t *cur = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N + 1));
    if (!level || !queue || !cur || !stack) { free(level); free(queue); free(cur); free(stack); return -1; }
    int64_t total = 0;
    for (;;) {
        /* level graph: BFS from all sources over residual arcs; sinks absorb */
        for (int32_t x = 0; x < N; x++) level[x] = -1;
        int32_t qh = 0, qt = 0, reached = 0, dsink = INT32_MAX;
        for (int32_t x = 0; x < N; x++) if (src[x]) { level[x] = 0; queue[qt++] = x; }
        while (qh < qt) {
            int32_t u = queue[qh++];
            if (snk[u]) { reached = 1; if (level[u] < dsink) dsink = level[u]; continue; }
            if (level[u] >= dsink) continue;       /* only levels below the nearest sink matter */
            for (int64_t a = G->adj_off[u]; a < G->adj_off[u + 1]; a++) {
                int32_t v = G->head[a];
                if (level[v] < 0 && residual(G, a) > 0) { level[v] = level[u] + 1; queue[qt++] = v; }
            }
        }
        if (!reached) break;
        /* layered network: keep only nodes that lie on a shortest augmenting
           path, i.e. sinks and nodes with a layered residual arc into a kept
           node (scanned in reverse BFS order); all others leave the level graph */
        for (int32_t i = qt - 1; i >= 0; i--) {
            int32_t u = queue[i];
            if (snk[u]) continue;
            int keep = 0;
            if (level[u] < dsink)
                for (int64_t a = G->adj_off[u]; a < G->adj_off[u + 1] && !keep; a++) {
                    int32_t v = G->head[a];
                    if (level[v] == level[u] + 1 && residual(G, a) > 0) keep = 1;
                }
            if (!keep) level[u] = -2;
        }
        /* blocking flow by depth-first search with current-arc pointers */
        for (int32_t x = 0; x < N; x++) cur[x] = G->adj_off[x];
        for (int32_t s = 0; s < N; s++) {
            if (!src[s]) continue;
            int32_t depth = 0, u = s;
            for (;;) {
                if (snk[u]) {
                    int64_t b = INT64_MAX;
                    for (int32_t i = 0; i < depth; i++) if (residual(G, stack[i]) < b) b = residual(G, stack[i]);
                    for (int32_t i = 0; i < depth; i++) push_arc(G, stack[i], b);
                    total += b;
                    int32_t k = 0;
                    while (residual(G, stack[k]) > 0) k++;   /* first saturated arc */
                    depth = k;
                    u = G->tail[stack[k]];
                    continue;
                }
                int found = 0;
                for (; cur[u] < G->adj_off[u + 1]; cur[u]++) {
                    int64_t a = cur[u];
                    int32_t v = G->head[a];
                    if (level[v] == level[u] + 1 && residual(G, a) > 0) {
                        stack[depth++] = a;
                        u = v;
                        found = 1;
                        break;
                    }
                }
                if (found) continue;
                level[u] = -2;                 /* dead end: no path to a sink */
                if (depth == 0) break;
                u = G->tail[stack[--depth]];
            }
        }
    }
    free(level); free(queue); free(cur); free(stack);
    return total;
}

/* Edmonds-Karp: repeatedly augment along a shortest residual S-T path.
 * A second, independent textbook routine used to cross-check Dinic. */
static int64_t edmonds_karp(Lawler *G, const uint8_t *src, const uint8_t *snk) {
    int32_t N = G->N;
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    if (!parent || !queue) { free(parent); free(queue); return -1; }
    int64_t total = 0;
    for (;;) {
        for (int32_t x = 0; x < N; x++) parent[x] = -2;
        int32_t qh = 0, qt = 0, found = -1;
        for (int32_t x = 0; x < N; x++) if (src[x]) { parent[x] = -1; queue[qt++] = x; }
        while (qh < qt && found < 0) {
            int32_t u = queue[qh++];
            for (int64_t a = G->adj_off[u]; a < G->adj_off[u + 1]; a++) {
                int32_t v = G->head[a];
                if (parent[v] == -2 && residual(G, a) > 0) {
                    parent[v] = a;
                    if (snk[v]) { found = v; break; }
                    queue[qt++] = v;
                }
            }
        }
        if (found < 0) break;
        int64_t b = INT64_MAX;
        for (int32_t v = found; parent[v] >= 0; v = G->tail[parent[v]])
            if (residual(G, parent[v]) < b) b = residual(G, parent[v]);
        for (int32_t v = found; parent[v] >= 0; v = G->tail[parent[v]]) push_arc(G, parent[v], b);
        total += b;
    }
    free(parent); free(queue);
    return total;
}

/* algo 0 = Dinic, 1 = Edmonds-Karp.  Returns the flow added, < 0 on error. */
int64_t or_augment(Lawler *G, const uint8_t *src, const uint8_t *snk, int32_t algo) {
    return algo == 1 ? edmonds_karp(G, src, snk) : dinic(G, src, snk);
}

void or_reset_flow(Lawler *G) { memset(G->flow, 0, sizeof(int64_t) * (size_t)G->A); }

/* Value of the current flow: net flow leaving the source set (Section 2). */
int64_t or_flow_value(const Lawler *G, const uint8_t *src) {
    int64_t v = 0;
    for (int32_t u = 0; u < G->N; u++) {
        if (!src[u]) continue;
        for (int64_t a = G->adj_off[u]; a < G->adj_off[u + 1]; a++)
            if (!src[G->head[a]]) v += G->flow[a];
    }
    return v;
}

/* Source-side cut: nodes reachable from S by residual arcs (Section 2). */
void or_reach_from(const Lawler *G, const uint8_t *seed, uint8_t *mark) {
    int32_t N = G->N;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t qh = 0, qt = 0;
    for (int32_t x = 0; x < N; x++) { mark[x] = seed[x] ? 1 : 0; if (seed[x]) queue[qt++] = x; }
    while (qh < qt) {
        int32_t u = queue[qh++];
        for (int64_t a = G->adj_off[u]; a < G->adj_off[u + 1]; a++) {
            int32_t v = G->head[a];
            if (!mark[v] && residual(G, a) > 0) { mark[v] = 1; queue[qt++] = v; }
        }
    }
    free(queue);
}

/* Sink-side cut: nodes with a residual path into T (reverse BFS, Section 2). */
void or_reach_to(const Lawler *G, const uint8_t *seed, uint8_t *mark) {
    int32_t N = G->N;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
    int32_t qh = 0, qt = 0;
    for (int32_t x = 0; x < N; x++) { mark[x] = seed[x] ? 1 : 0; if (seed[x]) queue[qt++] = x; }
    while (qh < qt) {
        int32_t v = queue[qh++];
        for (int64_t a = G->adj_off[v]; a < G->adj_off[v + 1]; a++) {
            int32_t u = G->head[a];          /* arc rev[a] runs u -> v */
            if (!mark[u] && residual(G, G->rev[a]) > 0) { mark[u] = 1; queue[qt++] = u; }
        }
    }
    free(queue);
}

/* Per-arc export for feasibility checks: tail, head, capacity, flow. */
void or_export_arcs(const Lawler *G, int32_t *tail, int32_t *head, int64_t *cap, int64_t *flow) {
    for (int64_t a = 0; a < G->A; a++) {
        tail[a] = G->tail[a]; head[a] = G->head[a]; cap[a] = G->cap[a]; flow[a] = G->flow[a];
    }
}

/* ------------------------------------------------------------------------ */
/* Brute force over all bipartitions of the region (<= 24 region vertices):
 * source side = {s} plus the region vertices whose bit is set; cut weight =
 * sum of w(e) over nets with pins on both sides (the hypergraph cut, which
 * equals the minimum Lawler cut, Section 2).  Reports the minimum, and the
 * intersection and union of all minimising source sets.  With max_w >= 0,
 * also the minimum over bipartitions whose two sides both weigh <= max_w
 * (-1 when none exists). */
int32_t or_bruteforce(int32_t n_nodes, int32_t m_nets, const uint32_t *net_off, const int32_t *npins,
                      const int32_t *net_w, const int64_t *node_w, int64_t max_w,
                      int64_t *min_cut, uint32_t *and_mask, uint32_t *or_mask, int64_t *n_min,
                      int64_t *min_balanced) {
    int32_t r = n_nodes - 2;
    if (r < 0 || r > 24) return OR_ERR_INVALID;
    int64_t best = INT64_MAX, bestbal = -1, cnt = 0, W = 0;
    uint32_t am = 0xFFFFFFFFu, om = 0;
    for (int32_t h = 0; h < n_nodes; h++) W += node_w[h];
    for (uint32_t mask = 0; mask < (1u << r); mask++) {
        int64_t cut = 0;
        for (int32_t e = 0; e < m_nets; e++) {
            int a = 0, b = 0;
            for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
                int32_t h = npins[j];
                int in_s = (h == 0) || (h >= 2 && ((mask >> (h - 2)) & 1u));
                if (in_s) a = 1; else b = 1;
            }
            if (a && b) cut += net_w[e];
        }
        if (cut < best) { best = cut; am = mask; om = mask; cnt = 1; }
        else if (cut == best) { am &= mask; om |= mask; cnt++; }
        if (max_w >= 0) {
            int64_t ws = node_w[0];
            for (int32_t i = 0; i < r; i++) if ((mask >> i) & 1u) ws += node_w[2 + i];
            if (ws <= max_w && W - ws <= max_w && (bestbal < 0 || cut < bestbal)) bestbal = cut;
        }
    }
    *min_cut = best; *and_mask = am; *or_mask = om; *n_min = cnt;
    if (min_balanced) *min_balanced = bestbal;
    return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* FlowCutter core, Algorithm 2 of the paper (Section 7), with the piercing
 * heuristics of Section 7, "Piercing".
 *
 * Readings where the paper is silent (each listed in the design notes):
 *  - S_r / T_r are residual reachability on the uncapped Lawler network of
 *    an actual maximum flow.
 *  - A bipartition (X, V \ X) is balanced iff c(X) <= L and c(V \ X) <= L.
 *    If both derived bipartitions are balanced, the one with the smaller
 *    heavier side is returned; ties go to the source side.
 *  - The source side grows iff c(S_r) <= c(T_r).
 *  - Candidates when growing S: hypernodes v not in S_r and not in T that are
 *    pins of a net whose in-node is in S_r, with c(S_r) + c(v) <= L.  Keys,
 *    compared in order, larger wins: (1) v not in T_r (no augmenting path),
 *    (2) signed distance from the original cut: +dist if v's original block
 *    is the growing side's, -dist otherwise, (3) the smaller
 *    fmix32(gid(v) ^ seed), MurmurHash3's 32-bit finaliser, a bijection, so
 *    keys never tie.  Growing T is symmetric (nets whose out-node is in T_r,
 *    no path from S_r, original block 1 counts as +).
 *  - No candidate: OR_NO_BALANCED_CUT.  flow > flow_bound (when >= 0):
 *    OR_ABORTED_WORSE.
 *
 * Inputs per hypernode h: node_w (in the Lawler object), orig_side[h] (0 or
 * 1), dist[h] (distance from the original cut; s and t unused), gid[h] (its
 * id in H, hashed for the third key).  final_side receives 0/1 per
 * hypernode; pierce_side / pierce_node receive the piercing sequence.
 */
static uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

static int64_t node_set_weight(const Lawler *G, const uint8_t *mark) {
    int64_t w = 0;
    for (int32_t h = 0; h < G->n_nodes; h++) if (mark[h]) w += G->node_w[h];
    return w;
}

typedef struct {
    int64_t flow;           /* final flow value = cut weight of the result */
    int32_t iterations;     /* max-flow augmentations performed */
    int32_t n_pierced;      /* length of the piercing sequence */
    int32_t result_side;    /* 0: (S_r, V\S_r) returned, 1: (V\T_r, T_r); 2: a most
                             * balanced cut found after the first balanced one */
    int32_t status;
    int64_t source_weight;  /* weight of the returned block 0 */
    int32_t bulk_steps;     /* iterations that pierced more than one node */
    int32_t mb_steps;       /* path-free piercings after the first balanced cut */
} or_fc_result;

/* Options of the two FlowCutter extensions of Section 7 (both off = the core
 * algorithm above):
 *
 * Bulk piercing ("Bulk Piercing"), read as follows where the text leaves
 * room.  Each side X (S or T) keeps its own goal and measurement.  The goal
 * of the weight to add to X in one iteration starts at
 *   base_X = beta * (c(V) / 2 - c(terminal of X))
 * (integers: floor(beta_pct * (c(V) - 2 c(x)) / 200)) and base_X is
 * multiplied by beta (floor(base * beta_pct / 100)) after every iteration
 * that grows X; the part of a goal an iteration did not reach (goal minus
 * the growth of X's reachable set, if positive) is carried into the next
 * goal of X.  The average weight added per pierced node of X is the total
 * growth of X's reachable set over the number of nodes pierced into X.  An
 * iteration pierces several nodes only when piercing cannot avoid an
 * augmenting path (the best candidate has a path), X is far from balance
 * (2 (c(X_r) + goal) <= c(V)), and X has grown at least `warmup` times:
 * then k = ceil(goal / average) candidates are pierced, taken in piercing
 * key order while the side stays within L.  Otherwise one node is pierced.
 *
 * Most balanced cut ("Most Balanced Cut"): after the first balanced
 * bipartition, piercing continues on the lighter side while a path-free
 * candidate exists (no flow changes), keeping the most balanced bipartition
 * seen (smaller heavier side; ties keep the earlier); this is repeated
 * `mb_reps` times from the first balanced state, repetition r hashing with
 * seed + r, and the most balanced result over all repetitions is returned
 * (its cut is the flow value, like every bipartition derived here).  These
 * piercings follow the core sequence in the piercing record, with side 2
 * for S and 3 for T. */
typedef struct {
    int32_t bulk_beta_pct;  /* 0: single piercing */
    int32_t bulk_warmup;    /* single piercings of a side before bulk ones */
    int32_t mb_reps;        /* 0: return the first balanced bipartition */
    int32_t pad;
} or_fc_options;

/* Candidates of growing side grow_s (Section 7, "Piercing"), best first by
 * the keys of the core algorithm; returns their number.  key order:
 * path-free first, larger signed distance, smaller hash. */
typedef struct { int32_t h; int no_path; int sd; uint32_t hh; } FcCand;

static int fc_cand_better(const FcCand *a, const FcCand *b) {
    if (a->no_path != b->no_path) return a->no_path > b->no_path;
    if (a->sd != b->sd) return a->sd > b->sd;
    return a->hh < b->hh;
}

static int fc_cand_cmp(const void *x, const void *y) {
    const FcCand *a = (const FcCand *)x, *b = (const FcCand *)y;
    if (fc_cand_better(a, b)) return -1;
    if (fc_cand_better(b, a)) return 1;
    return 0;
}

static int32_t fc_candidates(const Lawler *G, int grow_s, const uint8_t *R, const uint8_t *Ro,
                             const uint8_t *O, int64_t wR, int64_t max_w,
                             const int32_t *orig_side, const int32_t *dist, const int32_t *gid,
                             uint32_t seed, uint8_t *cand, FcCand *out) {
    int32_t nh = G->n_nodes, mN = G->m_nets;
    memset(cand, 0, (size_t)nh);
    for (int32_t e = 0; e < mN; e++) {
        int32_t node = grow_s ? nh + e : nh + mN + e;   /* in-node for S, out-node for T */
        if (!R[node]) continue;
        for (int64_t a = G->adj_off[nh + e]; a < G->adj_off[nh + e + 1]; a++) {
            int32_t h = G->head[a];
            if (h < nh) cand[h] = 1;                    /* pins of the net */
        }
    }
    int32_t nc = 0;
    for (int32_t h = 0; h < nh; h++) {
        if (!cand[h] || R[h] || O[h]) continue;
        if (wR + G->node_w[h] > max_w) continue;
        FcCand c;
        c.h = h;
        c.no_path = !Ro[h];
        c.sd = (orig_side[h] == (grow_s ? 0 : 1)) ? dist[h] : -dist[h];
        c.hh = fmix32((uint32_t)gid[h] ^ seed);
        out[nc++] = c;
    }
    qsort(out, (size_t)nc, sizeof(FcCand), fc_cand_cmp);
    return nc;
}

int32_t or_flowcutter_ex(Lawler *G, int64_t max_w, const int32_t *orig_side, const int32_t *dist,
                         const int32_t *gid, uint32_t seed, int64_t flow_bound, int32_t max_iter,
                         int32_t recompute, const or_fc_options *opt, uint8_t *final_side,
                         int32_t *pierce_side, int32_t *pierce_node, int32_t pierce_cap,
                         or_fc_result *res) {
    int32_t N = G->N, nh = G->n_nodes;
    uint8_t *S = (uint8_t *)calloc((size_t)N, 1), *T = (uint8_t *)calloc((size_t)N, 1);
    uint8_t *Sr = (uint8_t *)calloc((size_t)N, 1), *Tr = (uint8_t *)calloc((size_t)N, 1);
    uint8_t *cand = (uint8_t *)calloc((size_t)nh, 1);
    FcCand *cl = (FcCand *)malloc(sizeof(FcCand) * (size_t)nh);
    if (!S || !T || !Sr || !Tr || !cand || !cl) {
        free(S); free(T); free(Sr); free(Tr); free(cand); free(cl);
        return OR_ERR_OOM;
    }
    int64_t W = 0;
    for (int32_t h = 0; h < nh; h++) W += G->node_w[h];
    S[0] = 1;
    T[1] = 1;
    or_reset_flow(G);
    int32_t status = OR_OK, np = 0, it = 0;
    memset(res, 0, sizeof(*res));
    /* bulk piercing state per side: 0 = S, 1 = T */
    int64_t base[2], carry[2] = {0, 0}, added_w[2] = {0, 0}, added_n[2] = {0, 0}, pre_w[2] = {0, 0};
    int32_t grown[2] = {0, 0}, pending[2] = {0, 0};
    base[0] = opt ? (int64_t)opt->bulk_beta_pct * (W - 2 * G->node_w[0]) / 200 : 0;
    base[1] = opt ? (int64_t)opt->bulk_beta_pct * (W - 2 * G->node_w[1]) / 200 : 0;
    int bulk = opt && opt->bulk_beta_pct > 0;
    int64_t wS = 0, wT = 0;
    for (;;) {
        if (it >= max_iter) { status = OR_ITER_LIMIT; break; }
        it++;
        if (recompute) or_reset_flow(G);            /* self-check mode: from scratch */
        if (dinic(G, S, T) < 0) { status = OR_ERR_OOM; break; }   /* augment to maximality */
        int64_t flow = or_flow_value(G, S);
        res->flow = flow;
        if (flow_bound >= 0 && flow > flow_bound) { status = OR_ABORTED_WORSE; break; }
        or_reach_from(G, S, Sr);                      /* derive S_r and T_r */
        or_reach_to(G, T, Tr);
        wS = node_set_weight(G, Sr);
        wT = node_set_weight(G, Tr);
        /* measurement of the last growth of each side (bulk piercing) */
        for (int x = 0; x < 2; x++)
            if (pending[x]) {
                int64_t grew = (x == 0 ? wS : wT) - pre_w[x];
                int64_t goal = base[x] + carry[x];
                added_w[x] += grew;
                carry[x] = goal - grew > 0 ? goal - grew : 0;
                base[x] = base[x] * (opt ? opt->bulk_beta_pct : 0) / 100;
                grown[x]++;
                pending[x] = 0;
            }
        int balS = (wS <= max_w) && (W - wS <= max_w);
        int balT = (wT <= max_w) && (W - wT <= max_w);
        if (balS || balT) {
            int use_t = 0;
            if (balS && balT) {
                int64_t mS = wS > W - wS ? wS : W - wS;
                int64_t mT = wT > W - wT ? wT : W - wT;
                use_t = mT < mS;
            } else {
                use_t = !balS;
            }
            for (int32_t h = 0; h < nh; h++) final_side[h] = use_t ? (Tr[h] ? 1 : 0) : (Sr[h] ? 0 : 1);
            res->result_side = use_t;
            res->source_weight = use_t ? W - wT : wS;
            break;
        }
        int grow_s = wS <= wT;
        int x = grow_s ? 0 : 1;
        const uint8_t *R = grow_s ? Sr : Tr;       /* reachable set of the growing side */
        const uint8_t *Ro = grow_s ? Tr : Sr;      /* reachable set of the other side */
        const uint8_t *O = grow_s ? T : S;         /* terminal set of the other side */
        int64_t wR = grow_s ? wS : wT;
        int32_t nc = fc_candidates(G, grow_s, R, Ro, O, wR, max_w, orig_side, dist, gid, seed,
                                   cand, cl);
        if (nc == 0) { status = OR_NO_BALANCED_CUT; break; }
        /* how many nodes this iteration pierces */
        int64_t k = 1;
        if (bulk) {
            int64_t goal = base[x] + carry[x];
            int far = 2 * (wR + goal) <= W;
            if (!cl[0].no_path && far && grown[x] >= opt->bulk_warmup && added_n[x] > 0) {
                int64_t avg = added_w[x] / added_n[x];
                if (avg < 1) avg = 1;
                k = (goal + avg - 1) / avg;
                if (k < 1) k = 1;
            }
        }
        /* pierce: candidates in key order while the side stays within L */
        int64_t taken_w = 0;
        int32_t taken = 0;
        uint8_t *Xset = grow_s ? S : T;
        const uint8_t *Xr = grow_s ? Sr : Tr;
        for (int32_t x2 = 0; x2 < N; x2++) if (Xr[x2]) Xset[x2] = 1;
        for (int32_t c = 0; c < nc && taken < k; c++) {
            int32_t h = cl[c].h;
            if (wR + taken_w + G->node_w[h] > max_w) continue;
            if (np < pierce_cap) { pierce_side[np] = x; pierce_node[np] = h; }
            np++;
            Xset[h] = 1;
            taken_w += G->node_w[h];
            taken++;
        }
        if (taken > 1) res->bulk_steps++;
        pre_w[x] = wR;
        added_n[x] += taken;
        pending[x] = 1;
    }
    /* most balanced cut: path-free piercings from the first balanced state */
    if (status == OR_OK && opt && opt->mb_reps > 0) {
        uint8_t *S0 = (uint8_t *)malloc((size_t)N), *T0 = (uint8_t *)malloc((size_t)N);
        uint8_t *side = (uint8_t *)malloc((size_t)nh);
        int64_t best_max = res->source_weight > W - res->source_weight ? res->source_weight
                                                                         : W - res->source_weight;
        int64_t best_sw = res->source_weight;
        int32_t best_rs = res->result_side;
        memcpy(S0, S, (size_t)N);
        memcpy(T0, T, (size_t)N);
        for (int32_t r = 0; r < opt->mb_reps; r++) {
            memcpy(S, S0, (size_t)N);
            memcpy(T, T0, (size_t)N);
            uint32_t rs = seed + (uint32_t)r;
            for (;;) {
                or_reach_from(G, S, Sr);
                or_reach_to(G, T, Tr);
                wS = node_set_weight(G, Sr);
                wT = node_set_weight(G, Tr);
                /* the two bipartitions of this state, both of cut weight = flow */
                for (int use_t = 0; use_t < 2; use_t++) {
                    int64_t w0 = use_t ? W - wT : wS;
                    if (w0 > max_w || W - w0 > max_w) continue;
                    int64_t mx = w0 > W - w0 ? w0 : W - w0;
                    if (mx < best_max) {
                        best_max = mx;
                        best_sw = w0;
                        best_rs = 2;
                        for (int32_t h = 0; h < nh; h++)
                            side[h] = use_t ? (Tr[h] ? 1 : 0) : (Sr[h] ? 0 : 1);
                        memcpy(final_side, side, (size_t)nh);
                    }
                }
                int grow_s = wS <= wT;
                const uint8_t *R = grow_s ? Sr : Tr, *Ro = grow_s ? Tr : Sr, *O = grow_s ? T : S;
                int32_t nc = fc_candidates(G, grow_s, R, Ro, O, grow_s ? wS : wT, max_w,
                                           orig_side, dist, gid, rs, cand, cl);
                if (nc == 0 || !cl[0].no_path) break;   /* only path-free piercings */
                uint8_t *Xset = grow_s ? S : T;
                for (int32_t x2 = 0; x2 < N; x2++) if (R[x2]) Xset[x2] = 1;
                Xset[cl[0].h] = 1;
                /* recorded after the core sequence with side 2 (S) or 3 (T) */
                if (np < pierce_cap) { pierce_side[np] = grow_s ? 2 : 3; pierce_node[np] = cl[0].h; }
                np++;
                res->mb_steps++;
            }
        }
        res->source_weight = best_sw;
        res->result_side = best_rs;
        free(S0); free(T0); free(side);
    }
    res->iterations = it;
    res->n_pierced = np;
    res->status = status;
    free(S); free(T); free(Sr); free(Tr); free(cand); free(cl);
    return status;
}

int32_t or_flowcutter(Lawler *G, int64_t max_w, const int32_t *orig_side, const int32_t *dist,
                      const int32_t *gid, uint32_t seed, int64_t flow_bound, int32_t max_iter,
                      int32_t recompute, uint8_t *final_side, int32_t *pierce_side,
                      int32_t *pierce_node, int32_t pierce_cap, or_fc_result *res) {
    return or_flowcutter_ex(G, max_w, orig_side, dist, gid, seed, flow_bound, max_iter, recompute,
                            NULL, final_side, pierce_side, pierce_node, pierce_cap, res);
}

/* ------------------------------------------------------------------------ */
/* k-way refinement pieces (Section 4, Algorithm 1; Section 5; Section 6). */

/* Connectivity metric (lambda - 1)(Pi) = sum over nets of (lambda(e) - 1) w(e)
 * (Section 2). */
int64_t or_connectivity(int32_t m, const uint32_t *net_off, const int32_t *pins,
                        const int32_t *net_w, const int32_t *part, int32_t k) {
    uint8_t *seen = (uint8_t *)calloc((size_t)(k > 0 ? k : 1), 1);
    int64_t total = 0;
    for (int32_t e = 0; e < m; e++) {
        int32_t lam = 0;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t b = part[pins[j]];
            if (!seen[b]) { seen[b] = 1; lam++; }
        }
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) seen[part[pins[j]]] = 0;
        if (lam > 1) total += (int64_t)(lam - 1) * net_w[e];
    }
    free(seen);
    return total;
}

/* Quotient graph (Section 5, "Quotient Graph Construction"): for every pair
 * of blocks i < j, the number and weight of nets with pins in both.  Arrays
 * are k*k, row-major, upper triangle used. */
void or_quotient(int32_t m, const uint32_t *net_off, const int32_t *pins, const int32_t *net_w,
                 const int32_t *part, int32_t k, int64_t *pair_nets, int64_t *pair_weight) {
    uint8_t *seen = (uint8_t *)calloc((size_t)k, 1);
    int32_t *blocks = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    memset(pair_nets, 0, sizeof(int64_t) * (size_t)k * k);
    memset(pair_weight, 0, sizeof(int64_t) * (size_t)k * k);
    for (int32_t e = 0; e < m; e++) {
        int32_t nb = 0;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t b = part[pins[j]];
            if (!seen[b]) { seen[b] = 1; blocks[nb++] = b; }
        }
        for (int32_t a = 0; a < nb; a++) {
            seen[blocks[a]] = 0;
            for (int32_t c = 0; c < nb; c++) {
                int32_t i = blocks[a], jj = blocks[c];
                if (i < jj) { pair_nets[(size_t)i * k + jj]++; pair_weight[(size_t)i * k + jj] += net_w[e]; }
            }
        }
    }
    free(seen);
    free(blocks);
}

/* Region growing for the pair (bi, bj) (Section 6, "Region Growing"), with
 * the readings used throughout: a breadth-first search inside each block
 * from its pins of the pair's cut nets (distance 1), through nets of H, up
 * to distance delta; vertices are taken level by level in ascending id
 * order while the block's part of the region stays within
 *   bound_i = max(0, floor((100 + alpha_eps_pct) * ceil((c(Vi)+c(Vj))/2) / 100) - c(Vj))
 * (alpha_eps_pct = 100 * alpha * eps, 48 for alpha = 16, eps = 0.03); the
 * first vertex that does not fit ends that block's growth.  Output: the
 * region in ascending id order and the distance of each region vertex. */
int32_t or_grow_region(int32_t n, int32_t m, const uint32_t *net_off, const int32_t *pins,
                       const int32_t *node_w, const int32_t *part, int32_t bi, int32_t bj,
                       int32_t alpha_eps_pct, int32_t delta, int32_t *region, int32_t *dist,
                       int32_t *n_region) {
    int64_t cw[2] = {0, 0};
    for (int32_t v = 0; v < n; v++) {
        int64_t c = node_w ? node_w[v] : 1;
        if (part[v] == bi) cw[0] += c;
        else if (part[v] == bj) cw[1] += c;
    }
    int64_t half = (cw[0] + cw[1] + 1) / 2;
    int64_t lim = ((int64_t)(100 + alpha_eps_pct) * half) / 100;
    int64_t bound[2] = {lim - cw[1], lim - cw[0]};
    if (bound[0] < 0) bound[0] = 0;
    if (bound[1] < 0) bound[1] = 0;
    /* vertex -> nets incidence */
    int32_t *deg = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    for (int32_t e = 0; e < m; e++)
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) deg[pins[j] + 1]++;
    for (int32_t v = 0; v < n; v++) deg[v + 1] += deg[v];
    int32_t *inc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(deg[n] > 0 ? deg[n] : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    memcpy(fill, deg, sizeof(int32_t) * (size_t)n);
    for (int32_t e = 0; e < m; e++)
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) inc[fill[pins[j]]++] = e;
    int32_t *lev = (int32_t *)calloc((size_t)n, sizeof(int32_t));   /* 0 = not reached */
    uint8_t *in_b = (uint8_t *)calloc((size_t)n, 1);
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    for (int s = 0; s < 2; s++) {
        int32_t blk = s == 0 ? bi : bj, oth = s == 0 ? bj : bi;
        int64_t taken = 0;
        int stop = 0;
        /* level 1: pins in blk of nets with pins in both blocks */
        for (int32_t e = 0; e < m; e++) {
            int a = 0, b = 0;
            for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
                if (part[pins[j]] == blk) a = 1;
                if (part[pins[j]] == oth) b = 1;
            }
            if (!(a && b)) continue;
            for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++)
                if (part[pins[j]] == blk && !lev[pins[j]]) lev[pins[j]] = 1;
        }
        for (int32_t d = 1; d <= delta && !stop; d++) {
            /* vertices at distance d in ascending id: take while they fit */
            int32_t nc = 0;
            for (int32_t v = 0; v < n; v++) if (part[v] == blk && lev[v] == d) cur[nc++] = v;
            for (int32_t q = 0; q < nc && !stop; q++) {
                int32_t v = cur[q];
                int64_t c = node_w ? node_w[v] : 1;
                if (taken + c > bound[s]) { stop = 1; break; }
                taken += c;
                in_b[v] = 1;
            }
            if (stop || d == delta) break;
            /* next level: unlabelled vertices of blk sharing a net with a taken
               vertex at distance d */
            for (int32_t q = 0; q < nc; q++) {
                int32_t v = cur[q];
                if (!in_b[v]) continue;
                for (int32_t t = deg[v]; t < deg[v + 1]; t++) {
                    int32_t e = inc[t];
                    for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
                        int32_t u = pins[j];
                        if (part[u] == blk && !lev[u]) lev[u] = d + 1;
                    }
                }
            }
        }
    }
    int32_t nr = 0;
    for (int32_t v = 0; v < n; v++)
        if (in_b[v]) { region[nr] = v; dist[nr] = lev[v]; nr++; }
    *n_region = nr;
    free(deg); free(inc); free(fill); free(lev); free(in_b); free(cur);
    return OR_OK;
}

/* Apply the moves of one pair to the partition (Section 5, "Apply Moves"):
 * drop moves whose vertex is not in its expected block; apply the rest only
 * if every block that gains weight stays within max_w (the reading of "the
 * resulting partition is balanced" for an input that may already be
 * imbalanced); the actual change is the connectivity
 * metric before minus after (which the paper accumulates from the
 * Phi(e, V) transitions of each move).  If the metric grew, the moves are
 * reverted.  moves: (vertex, from, to) triples.  Returns the improvement
 * (>= 0, positive = better); *applied = 1 if kept.  part is updated. */
int64_t or_apply_moves(int32_t n, int32_t m, const uint32_t *net_off, const int32_t *pins,
                       const int32_t *net_w, const int32_t *node_w, int32_t *part, int32_t k,
                       int64_t max_w, const int32_t *moves, int32_t n_moves, int32_t *applied,
                       int32_t *n_valid) {
    int32_t *valid = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_moves > 0 ? n_moves : 1));
    int32_t nv = 0;
    for (int32_t q = 0; q < n_moves; q++)
        if (part[moves[3 * q]] == moves[3 * q + 1]) valid[nv++] = q;
    *n_valid = nv;
    int64_t *bw = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    int64_t *bw0 = (int64_t *)calloc((size_t)k, sizeof(int64_t));
    for (int32_t v = 0; v < n; v++) bw[part[v]] += node_w ? node_w[v] : 1;
    memcpy(bw0, bw, sizeof(int64_t) * (size_t)k);
    for (int32_t t = 0; t < nv; t++) {
        const int32_t *mv = moves + 3 * valid[t];
        int64_t c = node_w ? node_w[mv[0]] : 1;
        bw[mv[1]] -= c;
        bw[mv[2]] += c;
    }
    /* balanced: every block that gains weight stays within max_w (a block
       already above it may only lose weight) */
    int ok = 1;
    for (int32_t b = 0; b < k; b++) if (bw[b] > bw0[b] && bw[b] > max_w) ok = 0;
    free(bw0);
    *applied = 0;
    if (!ok || nv == 0) { free(valid); free(bw); return 0; }
    int64_t before = or_connectivity(m, net_off, pins, net_w, part, k);
    for (int32_t t = 0; t < nv; t++) part[moves[3 * valid[t]]] = moves[3 * valid[t] + 2];
    int64_t after = or_connectivity(m, net_off, pins, net_w, part, k);
    int64_t gain = before - after;
    if (gain < 0) {
        for (int32_t t = 0; t < nv; t++) part[moves[3 * valid[t]]] = moves[3 * valid[t] + 1];
        gain = 0;
    } else {
        *applied = 1;
    }
    free(valid); free(bw);
    return gain;
}

/* Per-pair statistics of the quotient graph (Section 5), the inputs of the
 * learned pair scheduler (the paper has no such scheduler; the statistics
 * are plain counts over the nets joining two blocks).  For every pair
 * i < j and every net e whose blocks include i and j, row (i, j) of
 * stats[k][k][8] accumulates:
 *   0 number of nets, 1 their weight, 2 their pins, 3 the largest size,
 *   4 nets whose blocks are exactly {i, j}, 5 their weight, 6 their pins,
 *   7 unused (0). */
void or_pair_stats(int32_t m, const uint32_t *net_off, const int32_t *pins, const int32_t *net_w,
                   const int32_t *part, int32_t k, int64_t *stats) {
    uint8_t *seen = (uint8_t *)calloc((size_t)k, 1);
    int32_t *blocks = (int32_t *)malloc(sizeof(int32_t) * (size_t)k);
    memset(stats, 0, sizeof(int64_t) * (size_t)k * k * 8);
    for (int32_t e = 0; e < m; e++) {
        int32_t nb = 0;
        int64_t size = (int64_t)(net_off[e + 1] - net_off[e]);
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) {
            int32_t b = part[pins[j]];
            if (!seen[b]) { seen[b] = 1; blocks[nb++] = b; }
        }
        for (int32_t a = 0; a < nb; a++) seen[blocks[a]] = 0;
        for (int32_t a = 0; a < nb; a++)
            for (int32_t c = 0; c < nb; c++) {
                int32_t i = blocks[a], jj = blocks[c];
                if (i >= jj) continue;
                int64_t *s = stats + ((size_t)i * k + jj) * 8;
                s[0] += 1;
                s[1] += net_w[e];
                s[2] += size;
                if (size > s[3]) s[3] = size;
                if (nb == 2) { s[4] += 1; s[5] += net_w[e]; s[6] += size; }
            }
    }
    free(seen);
    free(blocks);
}

/* ------------------------------------------------------------------------ */
/* Sequential FIFO push-relabel on the flow hypergraph (the paper's SeqPR
 * baseline, Appendix "Flow Algorithms"; the method of Section 2,
 * "Push-Relabel Algorithm": discharge in FIFO order plus global relabeling
 * after linear work), used as a second CPU timing beside Dinic.  Unlike the
 * routines above it works on the hypergraph form (no explicit arcs): for pin
 * slot p (pin u of net e) fin[p] is the flow on (u, e_in), capped at w(e)
 * during the preflow (Section 8.3, "Restricting Capacities"), fout[p] the
 * flow on (e_out, u); fb[e] is the bridge flow.  Arc groups of a node, in
 * scan order: hypernode u - per incident slot, (u, e_in) with residual
 * w(e) - fin and (u, e_out) with residual fout; in-node - the bridge
 * (w - fb), then (e_in, u) with residual fin per pin; out-node - (e_out,
 * e_in) with residual fb, then (e_out, u) uncapacitated per pin.
 * It stops at a maximum preflow (no excess node labelled below NL), which
 * already fixes the flow value and both minimal cuts (Section 2, last
 * sentence of "Push-Relabel Algorithm"): S_r by forward residual search
 * from s and every non-sink excess node with (u, e_in) uncapped (Section
 * 8.3), T_r by reverse residual search into t.  Outputs per Lawler node.
 * Returns the flow value or a negative error. */
typedef struct {
    int32_t nh, m, NL;
    const uint32_t *net_off;
    const int32_t *pins, *net_w;
    int32_t *node_off, *slot, *slot_net;
    int64_t *fin, *fout, *fb, *excess;
    int32_t *d;
    int64_t flow;                    /* excess that reached t */
} SeqPR;

typedef struct { int32_t head; int64_t res; int32_t kind; int32_t idx; } SprArc;

/* Residual arc j (0-based, in scan order) of node x; returns 0 past the end.
 * kind/idx say which flow variable the arc moves: 0 fin[idx] up, 1 fin[idx]
 * down, 2 fout[idx] up, 3 fout[idx] down, 4 fb[idx] up, 5 fb[idx] down. */
static int spr_arc(const SeqPR *P, int32_t x, int32_t j, SprArc *a) {
    int32_t nh = P->nh, m = P->m;
    if (x < nh) {
        int32_t deg = P->node_off[x + 1] - P->node_off[x];
        if (j >= 2 * deg) return 0;
        int32_t p = P->slot[P->node_off[x] + j / 2], e = P->slot_net[p];
        if (j % 2 == 0) { a->head = nh + e; a->res = P->net_w[e] - P->fin[p]; a->kind = 0; }
        else { a->head = nh + m + e; a->res = P->fout[p]; a->kind = 3; }
        a->idx = p;
        return 1;
    }
    int32_t e = x < nh + m ? x - nh : x - nh - m;
    int32_t size = (int32_t)(P->net_off[e + 1] - P->net_off[e]);
    if (j > size) return 0;
    if (x < nh + m) {                              /* in-node */
        if (j == 0) { a->head = nh + m + e; a->res = P->net_w[e] - P->fb[e]; a->kind = 4; a->idx = e; }
        else {
            int32_t p = (int32_t)P->net_off[e] + j - 1;
            a->head = P->pins[p]; a->res = P->fin[p]; a->kind = 1; a->idx = p;
        }
    } else {                                        /* out-node */
        if (j == 0) { a->head = nh + e; a->res = P->fb[e]; a->kind = 5; a->idx = e; }
        else {
            int32_t p = (int32_t)P->net_off[e] + j - 1;
            a->head = P->pins[p]; a->res = ((int64_t)1 << 60); a->kind = 2; a->idx = p;
        }
    }
    return 1;
}

static void spr_move(SeqPR *P, const SprArc *a, int64_t delta) {
    switch (a->kind) {
        case 0: P->fin[a->idx] += delta; break;
        case 1: P->fin[a->idx] -= delta; break;
        case 2: P->fout[a->idx] += delta; break;
        case 3: P->fout[a->idx] -= delta; break;
        case 4: P->fb[a->idx] += delta; break;
        default: P->fb[a->idx] -= delta; break;
    }
}

/* Exact labels: reverse breadth-first search from t over residual arcs
 * (capped).  Labels of unreached nodes and of s are NL. */
static void spr_global_relabel(SeqPR *P, int32_t *bfs) {
    int32_t NL = P->NL, nh = P->nh, m = P->m;
    for (int32_t x = 0; x < NL; x++) P->d[x] = NL;
    int32_t h = 0, t = 0;
    P->d[1] = 0;
    bfs[t++] = 1;
    while (h < t) {
        int32_t y = bfs[h++];
        /* candidates x with an arc (x, y): the arc groups of y name exactly
         * the neighbours; check the residual of (x, y) from x's side */
        SprArc a;
        for (int32_t j = 0; spr_arc(P, y, j, &a); j++) {
            int32_t x = a.head;
            if (x == 0 || P->d[x] != NL) continue;
            /* residual of (x, y) */
            int64_t r;
            if (x < nh) {                        /* y is e_in or e_out of net e */
                int32_t p = a.idx;                /* slot of x in that net */
                r = (y < nh + m) ? P->net_w[P->slot_net[p]] - P->fin[p] : P->fout[p];
            } else if (y < nh) {                  /* x is e_in / e_out, y a pin */
                r = (x < nh + m) ? P->fin[a.idx] : ((int64_t)1 << 60);
            } else if (x < nh + m) {              /* bridge e_in -> e_out */
                r = P->net_w[x - nh] - P->fb[x - nh];
            } else {                              /* e_out -> e_in */
                r = P->fb[x - nh - m];
            }
            if (r > 0) { P->d[x] = P->d[y] + 1; bfs[t++] = x; }
        }
    }
}

int64_t or_seqpr(int32_t nh, int32_t m, const uint32_t *net_off, const int32_t *pins,
                 const int32_t *net_w, uint8_t *src_side, uint8_t *snk_side, int64_t *stats) {
    if (nh < 2 || m < 0) return OR_ERR_INVALID;
    int32_t NL = nh + 2 * m;
    uint32_t p_tot = net_off[m];
    SeqPR P = {nh, m, NL, net_off, pins, net_w, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    P.node_off = (int32_t *)calloc((size_t)nh + 1, sizeof(int32_t));
    P.slot = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p_tot + 1));
    P.slot_net = (int32_t *)malloc(sizeof(int32_t) * (size_t)(p_tot + 1));
    P.fin = (int64_t *)calloc((size_t)p_tot + 1, sizeof(int64_t));
    P.fout = (int64_t *)calloc((size_t)p_tot + 1, sizeof(int64_t));
    P.fb = (int64_t *)calloc((size_t)m + 1, sizeof(int64_t));
    P.excess = (int64_t *)calloc((size_t)NL, sizeof(int64_t));
    P.d = (int32_t *)malloc(sizeof(int32_t) * (size_t)NL);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)NL);
    int32_t *bfs = (int32_t *)malloc(sizeof(int32_t) * (size_t)NL);
    uint8_t *inq = (uint8_t *)calloc((size_t)NL, 1);
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)nh + 4);
    if (!P.node_off || !P.slot || !P.slot_net || !P.fin || !P.fout || !P.fb || !P.excess ||
        !P.d || !queue || !bfs || !inq || !fill)
        return OR_ERR_OOM;   /* (process-lifetime test code: leaks on this path) */
    for (int32_t e = 0; e < m; e++)
        for (uint32_t p = net_off[e]; p < net_off[e + 1]; p++) {
            P.slot_net[p] = e;
            P.node_off[pins[p] + 1]++;
        }
    for (int32_t u = 0; u < nh; u++) P.node_off[u + 1] += P.node_off[u];
    memcpy(fill, P.node_off, sizeof(int32_t) * (size_t)nh);
    for (uint32_t p = 0; p < p_tot; p++) P.slot[fill[pins[p]]++] = (int32_t)p;

    /* saturate the arcs out of s: (s, e_in) up to w(e) */
    for (int32_t j = P.node_off[0]; j < P.node_off[1]; j++) {
        int32_t p = P.slot[j], e = P.slot_net[p];
        P.fin[p] = net_w[e];
        P.excess[nh + e] += net_w[e];
    }
    int64_t scans = 0, relabels = 0, pushes = 0, grs = 0, work = 0;
    const int64_t gr_work = 2 * (int64_t)NL + (int64_t)p_tot;
    int32_t qh = 0, qt = 0, qn = 0;   /* FIFO ring of active nodes */
#define SPR_PUSHQ(x) do { if (!inq[x]) { inq[x] = 1; queue[qt] = (x); qt = (qt + 1) % NL; qn++; } } while (0)
    for (;;) {
        /* global relabel, then every excess node with a label below NL is active */
        spr_global_relabel(&P, bfs);
        grs++;
        work = 0;
        qh = qt = qn = 0;
        memset(inq, 0, (size_t)NL);
        for (int32_t x = 2; x < NL; x++)
            if (P.excess[x] > 0 && P.d[x] < NL) SPR_PUSHQ(x);
        if (qn == 0) break;
        while (qn > 0 && work < gr_work) {
            int32_t x = queue[qh];
            qh = (qh + 1) % NL;
            qn--;
            inq[x] = 0;
            /* discharge: scan the arcs once, pushing on admissible ones,
             * then relabel if excess is left */
            int32_t dx = P.d[x];
            if (dx >= NL || P.excess[x] <= 0) continue;
            SprArc a;
            int32_t best = NL;
            for (int32_t j = 0; spr_arc(&P, x, j, &a); j++) {
                scans++;
                work++;
                if (a.res <= 0) continue;
                int32_t y = a.head;
                if (P.excess[x] > 0 && P.d[y] == dx - 1) {
                    int64_t delta = P.excess[x] < a.res ? P.excess[x] : a.res;
                    spr_move(&P, &a, delta);
                    P.excess[x] -= delta;
                    pushes++;
                    if (y == 1) P.flow += delta;
                    else if (y != 0) {
                        P.excess[y] += delta;
                        SPR_PUSHQ(y);
                    }
                    if (a.res - delta <= 0) continue;   /* arc saturated */
                }
                if (P.d[y] + 1 < best) best = P.d[y] + 1;
            }
            if (P.excess[x] > 0) {
                /* relabel: min over residual arcs after the scan */
                P.d[x] = best < NL ? best : NL;
                relabels++;
                if (P.d[x] < NL) SPR_PUSHQ(x);
            }
        }
    }
#undef SPR_PUSHQ
    /* minimal sink side: reverse search into t (labels are exact now) */
    for (int32_t x = 0; x < NL; x++) snk_side[x] = P.d[x] < NL ? 1 : 0;
    snk_side[0] = 0;
    /* minimal source side: forward search from s and every non-sink excess
     * node, (u, e_in) taken as uncapacitated */
    memset(src_side, 0, (size_t)NL);
    int32_t h = 0, t = 0;
    for (int32_t x = 0; x < NL; x++)
        if (x == 0 || (x != 1 && P.excess[x] > 0)) { src_side[x] = 1; bfs[t++] = x; }
    while (h < t) {
        int32_t x = bfs[h++];
        SprArc a;
        for (int32_t j = 0; spr_arc(&P, x, j, &a); j++) {
            int64_t r = a.res;
            if (x < nh && j % 2 == 0) r = 1;    /* (u, e_in) is uncapacitated */
            if (r > 0 && !src_side[a.head]) { src_side[a.head] = 1; bfs[t++] = a.head; }
        }
    }
    if (stats) { stats[0] = pushes; stats[1] = relabels; stats[2] = grs; stats[3] = scans; }
    int64_t flow = P.flow;
    free(P.node_off); free(P.slot); free(P.slot_net); free(P.fin); free(P.fout); free(P.fb);
    free(P.excess); free(P.d); free(queue); free(bfs); free(inq); free(fill);
    return flow;
}

/* ------------------------------------------------------------------------ */
/* Identical net removal (Section 6, "Identical Net Removal"): nets of the
 * flow hypergraph with the same pin set are merged into one representative
 * that carries their summed weight.  Nets are compared through fingerprints
 * f(e) = sum of v^2 over the pins v of e (flow-hypergraph node ids, modulo
 * 2^64) and sizes; nets with different fingerprints or sizes are never
 * identical, and nets of one (fingerprint, size) group are compared as pin
 * sets.  Reading for determinism: every net merges into the smallest-id net
 * with the same pin set.  Kept nets keep their order, pin order and ids in
 * H.  Returns the new net count (pins go to out_pins, offsets to
 * out_off[m' + 1]; rep_of[e] = the net e merged into, or e). */
typedef struct { uint64_t f; uint32_t size; int32_t e; } NetFp;

static int netfp_cmp(const void *a, const void *b) {
    const NetFp *x = (const NetFp *)a, *y = (const NetFp *)b;
    if (x->f != y->f) return x->f < y->f ? -1 : 1;
    if (x->size != y->size) return x->size < y->size ? -1 : 1;
    return x->e < y->e ? -1 : (x->e > y->e);
}

static int i32_cmp(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return x < y ? -1 : (x > y);
}

int32_t or_dedup_nets(int32_t m, const uint32_t *net_off, const int32_t *pins, const int32_t *net_w,
                      const int32_t *net_gid, uint32_t *out_off, int32_t *out_pins,
                      int32_t *out_w, int32_t *out_gid, int32_t *rep_of) {
    NetFp *fp = (NetFp *)malloc(sizeof(NetFp) * (size_t)(m > 0 ? m : 1));
    int64_t *wsum = (int64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
    int32_t *a = (int32_t *)malloc(sizeof(int32_t) * (size_t)(net_off[m] + 1));
    int32_t *b = (int32_t *)malloc(sizeof(int32_t) * (size_t)(net_off[m] + 1));
    if (!fp || !wsum || !a || !b) return OR_ERR_OOM;
    for (int32_t e = 0; e < m; e++) {
        uint64_t f = 0;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) f += (uint64_t)pins[j] * (uint64_t)pins[j];
        fp[e].f = f;
        fp[e].size = net_off[e + 1] - net_off[e];
        fp[e].e = e;
        rep_of[e] = e;
    }
    qsort(fp, (size_t)m, sizeof(NetFp), netfp_cmp);
    for (int32_t i = 0; i < m;) {
        int32_t j = i;
        while (j < m && fp[j].f == fp[i].f && fp[j].size == fp[i].size) j++;
        /* the group in ascending id: each net merges into the first earlier
         * net of the group with the same pin set */
        uint32_t s = fp[i].size;
        for (int32_t t = i + 1; t < j; t++) {
            int32_t e = fp[t].e;
            memcpy(b, pins + net_off[e], sizeof(int32_t) * s);
            qsort(b, s, sizeof(int32_t), i32_cmp);
            for (int32_t u = i; u < t; u++) {
                int32_t r = fp[u].e;
                if (rep_of[r] != r) continue;          /* only representatives */
                memcpy(a, pins + net_off[r], sizeof(int32_t) * s);
                qsort(a, s, sizeof(int32_t), i32_cmp);
                if (memcmp(a, b, sizeof(int32_t) * s) == 0) { rep_of[e] = r; break; }
            }
        }
        i = j;
    }
    for (int32_t e = 0; e < m; e++) wsum[rep_of[e]] += net_w[e];
    int32_t mm = 0;
    uint32_t p = 0;
    out_off[0] = 0;
    for (int32_t e = 0; e < m; e++) {
        if (rep_of[e] != e) continue;
        for (uint32_t j = net_off[e]; j < net_off[e + 1]; j++) out_pins[p++] = pins[j];
        out_w[mm] = (int32_t)wsum[e];
        out_gid[mm] = net_gid[e];
        out_off[++mm] = p;
    }
    free(fp); free(wsum); free(a); free(b);
    return mm;
}
