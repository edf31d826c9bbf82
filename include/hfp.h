/*
 * hfp: flow-based hypergraph refinement on one GB300 (sm_103a).
 *
 * C ABI of libhfp.so.  Operations follow Gottesbueren, Heuer and Sanders,
 * "Parallel Flow-Based Hypergraph Partitioning" (arXiv 2201.01556):
 *   - flow network construction of a region (Section 6),
 *   - maximum flow by synchronous push-relabel on the Lawler expansion
 *     (Sections 2 and 8),
 *   - minimal source-side / sink-side minimum cuts (Sections 2 and 8.4),
 *   - one FlowCutter pierce-and-augment step and the whole FlowCutter loop
 *     (Section 7, Algorithm 2).
 *
 * Conventions (all entry points):
 *   - Return an hfp_status: HFP_OK (0) or a negative code.  hfp_last_error()
 *     gives a message for the calling thread's last failure.
 *   - Inputs are borrowed for the duration of the call; the library copies
 *     what it keeps.  Handles (hfp_ctx, hfp_net) are owned by the library and
 *     released by their destroy call.
 *   - Array arguments live in host or device memory as the hfp_mem argument
 *     of the call says.  Device pointers must be on the context's device.
 *   - All ids are int32, weights are int32 (> 0); flow values and weight sums
 *     are int64.  The sum of all net weights and the sum of all vertex
 *     weights must each stay below 2^31.
 *   - Work runs on the context's stream.  Calls that return values to the
 *     host synchronise that stream.
 *   - There is no CPU fallback: every step runs in this library's kernels.
 *
 * Flow hypergraph numbering (used by every per-node input and output):
 *   hypernode 0 = s (region-external vertices of side 0, contracted),
 *   hypernode 1 = t (region-external vertices of side 1, contracted),
 *   hypernode 2 + i = region[i];
 *   Lawler node of hypernode h = h, of the in-node of net e = n_nodes + e,
 *   of the out-node of net e = n_nodes + m_nets + e.
 *   Nets keep the ascending order of their ids in H; a net's pins are its
 *   region pins in H's order, then s, then t.
 */
#ifndef HFP_H
#define HFP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t hfp_status;

#define HFP_OK 0
#define HFP_ERR_INVALID (-1)          /* malformed input (CSR, ids, weights, duplicates) */
#define HFP_ERR_OOM (-2)              /* device or host allocation failed */
#define HFP_ERR_CUDA (-3)             /* a CUDA call failed */
#define HFP_ERR_ITER_LIMIT (-4)       /* a bounded device loop or wait gave up */
#define HFP_NO_BALANCED_CUT (-5)      /* FlowCutter found no piercing candidate */
#define HFP_ABORTED_WORSE (-6)        /* flow exceeded the bound (Section 8.3, "Flow Value") */
#define HFP_ERR_BUFFER_TOO_SMALL (-7) /* an output capacity is too small */
#define HFP_ERR_STATE (-8)            /* call out of order (e.g. cut before max flow) */

typedef enum { HFP_MEM_HOST = 0, HFP_MEM_DEVICE = 1 } hfp_mem;

typedef struct hfp_ctx hfp_ctx;
typedef struct hfp_net hfp_net;

/* Hypergraph H = (V, E, c, w) as a net -> pins CSR (Section 2).
 * net_off[m + 1] (non-decreasing, net_off[0] = 0), pins[net_off[m]] with ids
 * in [0, n) and no repeated pin inside a net, net_w[m] > 0, node_w[n] > 0 or
 * NULL for unit weights. */
typedef struct {
  int32_t n;
  int32_t m;
  const uint32_t* net_off;
  const int32_t* pins;
  const int32_t* net_w;
  const int32_t* node_w;
} hfp_hypergraph;

/* Sizes of a built flow network. */
typedef struct {
  int32_t n_nodes;       /* hypernodes, including s and t */
  int32_t m_nets;        /* nets kept */
  int64_t p_pins;        /* pins, including s/t pins ("Lawler-network pins") */
  int32_t lawler_nodes;  /* n_nodes + 2 * m_nets */
  int32_t pad;
  int64_t total_weight;  /* c(V) of the nodes of the network, s and t included */
} hfp_net_info;

/* Counters of the device engine since the network was built. */
typedef struct {
  uint64_t rounds;           /* discharge rounds */
  uint64_t global_relabels;
  uint64_t gr_levels;        /* reverse-BFS levels over all global relabels */
  uint64_t items_hyper;      /* hypernode incidences scanned */
  uint64_t items_net;        /* net pins scanned */
  uint64_t node_visits;      /* list entries processed */
  uint64_t pushes;
  uint64_t engine_launches;  /* cooperative launches of the engine kernel */
  uint64_t engine_ns;        /* device time of those launches (CUDA events on the context stream) */
  uint64_t gr_queue_entries; /* queue entries of the queue-driven global relabels */
  uint64_t gr_queue_overflows;  /* such relabels redone level by level (queue full) */
} hfp_stats;

/* FlowCutter parameters (Section 7).  The two extensions of Section 7 are
 * off when their fields are 0 (the batched launch supports neither):
 *  - bulk piercing ("Bulk Piercing"): each side keeps a goal of weight to add
 *    per iteration, starting at floor(bulk_beta_pct * (c(V) - 2 c(terminal))
 *    / 200) and multiplied by bulk_beta_pct / 100 after every iteration that
 *    grows the side, plus the part of the last goal not reached; when the
 *    best candidate opens an augmenting path, the side is far from balance
 *    (2 (c(X_r) + goal) <= c(V)) and the side has grown bulk_warmup times,
 *    ceil(goal / average growth per pierced node) candidates are pierced at
 *    once, in piercing-key order while the side stays within L;
 *  - most balanced cut ("Most Balanced Cut"): after the first balanced
 *    bipartition, mb_reps repetitions (third key seeded with seed + r) of
 *    path-free piercings of the lighter side from that state; the most
 *    balanced bipartition seen (lighter heavier side, earlier on ties) is
 *    returned; these piercings follow the others in the piercing record with
 *    side 2 (S) or 3 (T). */
typedef struct {
  int64_t max_block_weight;  /* L: a side is balanced iff its weight <= L */
  int64_t flow_bound;        /* abort with HFP_ABORTED_WORSE once flow > bound; < 0: none */
  uint32_t seed;             /* seeds the third piercing key */
  int32_t max_iterations;    /* <= 0: no limit beyond the number of hypernodes */
  int32_t bulk_beta_pct;     /* bulk piercing's beta in percent; 0: off */
  int32_t bulk_warmup;       /* single piercings of a side before bulk ones */
  int32_t mb_reps;           /* most balanced cut repetitions (<= 1024); 0: off */
  int32_t pad;
} hfp_fc_params;

typedef struct {
  int64_t flow;              /* final flow = cut weight of the returned bipartition */
  int64_t source_weight;     /* weight of block 0 of the returned bipartition */
  int32_t iterations;        /* max-flow augmentations */
  int32_t n_pierced;         /* piercing steps taken */
  int32_t result_side;       /* 0: (S_r, V \ S_r) returned; 1: (V \ T_r, T_r);
                              * 2: a more balanced cut found after the first one */
  int32_t device_us;         /* batched launch: device time of this problem in its group
                              * (microseconds, globaltimer); 0 elsewhere */
  int32_t bulk_steps;        /* iterations that pierced several nodes */
  int32_t mb_steps;          /* path-free piercings of the most balanced cut search */
} hfp_fc_result;

/* --- context --------------------------------------------------------------
 * Creates a context on CUDA device `device`.  `stream` is a cudaStream_t
 * (NULL = the legacy default stream); the context does not own it. */
hfp_status hfp_ctx_create(hfp_ctx** ctx, int device, void* stream);
/* Releases the caller's handle; networks built from the context stay usable
 * and the context is freed with the last of them. */
void hfp_ctx_destroy(hfp_ctx* ctx);
/* Message of the calling thread's last failed call ("" if none). */
const char* hfp_last_error(void);
/* Number of kernels this library has launched in the process so far. */
uint64_t hfp_kernel_launches(void);

/* --- engine tuning -------------------------------------------------------------
 * Speed-only knobs of the flow engine; no value changes any result (flow,
 * hypernode cuts, piercing sequence).  Defaults in brackets.
 *   gr_work_x100  global relabel once the frontier and next-list entries
 *                 processed since the last one exceed gr_work_x100 / 100
 *                 Lawler nodes (Section 8.1, "after linear work") [200]
 *   stall_rounds, stall_nodes  also relabel globally after stall_rounds
 *                 rounds without a flow change, each with fewer than
 *                 stall_nodes active nodes (Section 8.3) [100, 1500]
 *   tail_enter, tail_exit  frontiers of at most tail_enter nodes are run by
 *                 one CTA with block barriers until they exceed tail_exit
 *                 [64, 192]
 *   max_rounds    discharge-round budget of one network [2^22]
 *   bfs_enter, bfs_exit  breadth-first-search levels (global relabel, S_r,
 *                 distances) of at most bfs_enter nodes (a heavy node counts
 *                 32) are run by one CTA until they exceed bfs_exit
 *                 [0, 0]: off; 0 still runs empty levels alone
 *   pierce_relabel  after a source-side piercing that creates an augmenting
 *                 path, start the flow with a global relabel instead of
 *                 rounds on the new excess (Section 8.4 skips it) [0]
 *   stall_rounds_pierce  the stall_rounds rule for the incremental flows
 *                 after a piercing; 0: adaptive, as many rounds as the last
 *                 global relabel had levels (at least 8, at most 200) [0]
 *   async_gr      global relabels of hfp_max_flow / hfp_flowcutter as one
 *                 label-correcting search driven by a device work queue,
 *                 without a grid barrier per breadth-first level; the labels
 *                 are the same exact distances [1]
 *   gr_warps      warps per CTA that serve that queue (1..16) [12]
 *   identical_nets  networks built from now on merge nets with identical pin
 *                 sets into the smallest-id one, which carries their summed
 *                 weight (Section 6, "Identical Net Removal"); flows, cut
 *                 sides over the hypernodes and FlowCutter outcomes are
 *                 unchanged, Lawler-node outputs and cut net ids refer to
 *                 the merged nets (representatives' ids in H) [0]
 *   fused_rounds  one grid-wide phase per discharge round: each node applies
 *                 the previous round's pushes, discharges and relabels itself
 *                 from its own residual arcs, raising its label by at most 2;
 *                 0: a push phase and a relabel phase per round [1]
 *   batch_cluster  batched FlowCutter: launch groups of at most 16 CTAs as
 *                 thread-block clusters (group barriers in distributed
 *                 shared memory) when as many such clusters can be resident
 *                 as there would be groups; 2: also when fewer can, with
 *                 only that many groups; 0: always one cooperative launch
 *                 with barriers in global memory.  With two CTAs per SM a
 *                 full grid of groups does not fit as clusters on GB300
 *                 (a GPC of ~19 SMs holds two 16-CTA clusters), so 1 runs
 *                 cooperative there [1]
 *   batch_big_ctas, batch_big_groups  batched FlowCutter: the first
 *                 batch_big_groups groups get batch_big_ctas CTAs each (the
 *                 largest problems start on them), the others the launch's
 *                 group size; used when batch_big_ctas exceeds that size
 *                 [0, 0]: uniform groups
 *   batch_fused_rounds, batch_async_gr  fused_rounds and async_gr for the
 *                 flows of the batched FlowCutter [1, 0]: in groups of a few
 *                 CTAs a level costs little more than its work, and the
 *                 queue-driven search measured slower there
 *   parpr_block   one-phase rounds keep labels valid by ParPR-Block
 *                 (Section 8.2, first fix: in a round a node pushed to may not
 *                 relabel and a relabeled node may not be pushed to, whichever
 *                 comes first) instead of capping a self relabel at d + 2 [0]
 *   construction  flow networks of k-way block pairs (Section 6,
 *                 "Construction Algorithms"): 1 scans the nets of the two
 *                 blocks; 2 sorts the region's (net, vertex) incidences by net;
 *                 0 takes 2 when |E| <= |V| / 2 or the average net has >= 100
 *                 pins, as the paper does, else 1.  The networks are the same.
 *                 Here the first algorithm only scans the nets of the two
 *                 blocks (per-round block lists), and it measured faster on
 *                 dense and sparse rings alike (8M: 251 vs 282 ms of pair
 *                 preparation per round; |E| = 0.4 |V|: 176 vs 205 ms) [1]
 *   batch_gr_work_x100, batch_stall_rounds_pierce  gr_work_x100 and
 *                 stall_rounds_pierce of the batched FlowCutter [100, 30]:
 *                 the engine autotuner picked both on the 1M and 8M k = 64
 *                 rounds (launch 1028 -> 950 ms and 2730 -> 2653 ms)
 *   wait_timeout_ms  bound on every device wait of this context's launches
 *                 (grid, group and cluster barriers, the relabel queue's
 *                 waits, one-CTA loops), 1..600000 ms; a wait that runs out
 *                 sets the launch's error word, every CTA leaves, and the
 *                 call returns HFP_ERR_ITER_LIMIT with the context usable
 *                 [10000]
 *   prep_streams  k-way rounds prepare their block pairs (region growing,
 *                 network construction; Section 6) on this many host threads
 *                 (1..16), each with a stream and region scratch of its own,
 *                 so that their host round trips overlap; 1: one after
 *                 another on the context's stream.  The networks are the
 *                 same.  Preparation of one round, 1 -> 8 threads: 8M
 *                 vertices 255 -> 99 ms, a 2M-vertex sparse ring 181 -> 49 ms
 *                 [8] */
typedef struct {
  uint32_t gr_work_x100;
  uint32_t stall_rounds;
  uint32_t stall_nodes;
  uint32_t tail_enter;
  uint32_t tail_exit;
  uint32_t max_rounds;
  uint32_t bfs_enter;
  uint32_t bfs_exit;
  uint32_t pierce_relabel;
  uint32_t stall_rounds_pierce;
  uint32_t batch_cluster;
  uint32_t batch_big_ctas;
  uint32_t batch_big_groups;
  uint32_t async_gr;
  uint32_t gr_warps;
  uint32_t fused_rounds;
  uint32_t identical_nets;
  uint32_t batch_fused_rounds;
  uint32_t batch_async_gr;
  uint32_t parpr_block;
  uint32_t construction;
  uint32_t batch_gr_work_x100;
  uint32_t batch_stall_rounds_pierce;
  uint32_t wait_timeout_ms;
  uint32_t prep_streams;
} hfp_tuning;
hfp_status hfp_ctx_get_tuning(hfp_ctx* ctx, hfp_tuning* tuning);
hfp_status hfp_ctx_set_tuning(hfp_ctx* ctx, const hfp_tuning* tuning);

/* --- network construction (Section 6, "Construction Algorithms") ---------
 * Builds the flow hypergraph of the region B = region[0 .. n_region):
 * every net of H with a pin in B is copied with its region pins; a pin
 * outside B whose side is 0 adds s, side 1 adds t (once per net); pins of any
 * other side are ignored.  Nets left with fewer than two pins, or holding
 * both s and t, are dropped (Section 6, end of "Construction Algorithms").
 *   H, region, side, dist_from_cut: in `mem` memory.
 *   side[n]: 0 or 1 for vertices of the two blocks, any other value for
 *            vertices outside both; every region vertex must have side 0/1.
 *   dist_from_cut[n_region]: distance of region[i] from the original cut,
 *            used by the piercing rule (Section 7, "Piercing"); NULL makes
 *            the library compute it: region pins of nets of H with pins on
 *            both sides get 1, unlabelled region pins of a net holding a
 *            region vertex at distance d get d + 1, unreached vertices
 *            2^20 - 1.
 * Errors: HFP_ERR_INVALID (ids out of range, repeated region vertex, region
 * vertex without side 0/1, non-positive weight, weight sums >= 2^31),
 * HFP_ERR_OOM, HFP_ERR_CUDA.  *out is NULL on error. */
hfp_status hfp_build_flow_network(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                                  const int32_t* region, int32_t n_region, const int32_t* side,
                                  const int32_t* dist_from_cut, hfp_net** out);
void hfp_net_destroy(hfp_net* net);
hfp_status hfp_net_get_info(hfp_net* net, hfp_net_info* info);
/* Copies the network CSR to caller buffers in `mem` memory (any pointer may
 * be NULL to skip it): net_off[m_nets + 1], pins[p_pins], net_w[m_nets],
 * net_gid[m_nets] (ids in H), node_w[n_nodes], node_off[n_nodes + 1] and
 * inc_slot[p_pins] (hypernode -> pin slots, ascending), dist[n_nodes]. */
hfp_status hfp_net_export(hfp_net* net, hfp_mem mem, uint32_t* net_off, int32_t* pins,
                          int32_t* net_w, int32_t* net_gid, int32_t* node_w, uint32_t* node_off,
                          int32_t* inc_slot, int32_t* dist);
hfp_status hfp_net_get_stats(hfp_net* net, hfp_stats* stats);
/* Copies the network's current (pre)flow to caller buffers in `mem` memory
 * (any pointer may be NULL to skip it), for checking it (Section 2,
 * "Flows": capacity and conservation; Section 8.3, "Restricting
 * Capacities": the cap f(u, e_in) <= w(e)):
 *   f_in[p_pins]   flow on (u, e_in) of each pin slot, 0 <= f_in <= w(e);
 *   f_out[p_pins]  flow on (e_out, u) of each pin slot, >= 0;
 *   f_b[m_nets]    flow on the bridge (e_in, e_out), 0 <= f_b <= w(e);
 *   excess[lawler_nodes]  excess of each non-terminal Lawler node (inflow -
 *                  outflow once every push of the last round is applied;
 *                  values of sources and sinks are not maintained);
 *   delta[lawler_nodes]   pushes not yet applied to excess, summed over
 *                  the engine's delta buffers (all 0 once hfp_max_flow
 *                  returned);
 *   flags[lawler_nodes]   bit 0: node is in S, bit 1: node is in T.
 * The flow value is the net inflow of T.  Per-arc flows are not unique;
 * only the value and the minimal cuts are. */
hfp_status hfp_net_export_flow(hfp_net* net, hfp_mem mem, int32_t* f_in, int32_t* f_out,
                               int32_t* f_b, int64_t* excess, int64_t* delta, uint8_t* flags);


/* --- tracing ----------------------------------------------------------------
 * hfp_net_enable_trace keeps a trace of the next `phases` engine phases
 * (allocates 32 bytes per phase on the device).  hfp_net_get_trace copies to
 * host memory: state_ns[10] / state_cnt[10], the device time (globaltimer)
 * spent in, and the number of, engine phases of each state (0 done, 1 push,
 * 2 relabel/apply, 3/4 global relabel init/level, 5/6 S_r init/level, 7/8
 * distance init/level, 9 phases run by one CTA); trace[4 * cap] holds four
 * words per phase: (state | one_cta << 5) << 58 | light input << 29 | heavy
 * input; light output << 32 | heavy output; the flow value; the phase's
 * device time in ns.  The input is the frontier (push), the next list
 * (relabel/apply) or the breadth-first-search level, the output the list the
 * phase filled.  *n = phases recorded. */
hfp_status hfp_net_enable_trace(hfp_net* net, int32_t phases);
hfp_status hfp_net_get_trace(hfp_net* net, uint64_t* state_ns, uint64_t* state_cnt,
                             uint64_t* trace, int32_t cap, int32_t* n);

/* --- maximum flow (Section 8) ---------------------------------------------
 * Augments the network's current flow to a maximum preflow with respect to
 * its current source set S and sink set T (initially {s} and {t}); on return
 * labels are exact distances to T, so the sink side T_r is known.  Returns
 * the flow value (excess that reached T).  HFP_ERR_ITER_LIMIT if the round
 * budget or a device wait ran out. */
hfp_status hfp_max_flow(hfp_net* net, int64_t* flow_value);

/* --- minimum cuts (Section 2; Section 8.4 "Source-Side Cut") -------------
 * Requires a completed hfp_max_flow.  The source side S_r is the set of
 * Lawler nodes reachable by residual arcs from S and from every non-sink
 * node with excess; it is the minimal source side of all minimum cuts.
 * Outputs (in `mem` memory, each may be NULL):
 *   in_source_lawler[lawler_nodes], in_source_region[n_region]: 1 if in S_r;
 *   cut_nets[cap]: ids in H of the nets whose in-node is in S_r and whose
 *   out-node is not (the cut nets), *n_cut their number
 *   (HFP_ERR_BUFFER_TOO_SMALL if cap < *n_cut; *n_cut is still set);
 *   *source_weight = c(S_r), the hypernode weight of S_r. */
hfp_status hfp_min_cut_source_side(hfp_net* net, hfp_mem mem, uint8_t* in_source_lawler,
                                   uint8_t* in_source_region, int32_t* cut_nets, int32_t cap,
                                   int32_t* n_cut, int64_t* source_weight);
/* Sink side T_r: Lawler nodes with a residual path into T (the minimal sink
 * side).  Outputs as above; *sink_weight = c(T_r). */
hfp_status hfp_min_cut_sink_side(hfp_net* net, hfp_mem mem, uint8_t* in_sink_lawler,
                                 uint8_t* in_sink_region, int64_t* sink_weight);

/* --- one FlowCutter step (Section 7, Algorithm 2 lines 7-10) -------------
 * side 0: S <- S_r + nodes; side 1: T <- T_r + nodes, then augments the flow
 * to maximality again (a source-side pierce keeps the labels; a sink-side
 * pierce adds the excess of the new sinks to the flow value and runs a
 * global relabel first, Section 8.4).  nodes[count] are hypernode ids in
 * host memory; nodes == NULL selects one node by the piercing rule (see
 * hfp_flowcutter) and stores it in *pierced.  Returns the new flow value.
 * HFP_NO_BALANCED_CUT when the rule finds no candidate. */
hfp_status hfp_pierce_and_augment(hfp_net* net, int32_t side, const int32_t* nodes,
                                  int32_t count, const hfp_fc_params* params, int32_t* pierced,
                                  int64_t* flow_value);

/* --- FlowCutter (Section 7, Algorithm 2) ----------------------------------
 * Runs max flow / cut derivation / piercing until (S_r, V \ S_r) or
 * (V \ T_r, T_r) is balanced (both sides <= L).  If both are, the one with
 * the lighter heavier side is returned (ties: the source side).  The lighter
 * reachable side grows (S on ties).  Piercing candidates for S are hypernodes
 * not in S_r and not in T that are pins of a net whose in-node is in S_r and
 * whose weight keeps c(S_r) + c(v) <= L; the best has, in order: no residual
 * path to T (v not in T_r); the larger signed distance from the original cut
 * (+dist if v's original side is 0, -dist otherwise); the smaller
 * fmix32(id_in_H(v) ^ seed).  T grows symmetrically.
 * Outputs (host memory, may be NULL): final_side[n_region] (0 = block of s),
 * pierce_side[pierce_cap] / pierce_node[pierce_cap] (hypernode ids), result.
 * Errors: HFP_NO_BALANCED_CUT, HFP_ABORTED_WORSE, HFP_ERR_ITER_LIMIT,
 * HFP_ERR_BUFFER_TOO_SMALL (pierce_cap too small; the run still completes). */
hfp_status hfp_flowcutter(hfp_net* net, const hfp_fc_params* params, uint8_t* final_side,
                          int32_t* pierce_side, int32_t* pierce_node, int32_t pierce_cap,
                          hfp_fc_result* result);

/* --- batched FlowCutter ---------------------------------------------------
 * hfp_flowcutter on n networks in ONE cooperative kernel launch.  The grid
 * is cut into groups of group_ctas CTAs (<= 0: as many CTAs per group as the
 * grid allows with one group per network); each group takes the next network
 * from a device work queue (largest first) and runs all of Algorithm 2 on it
 * without returning to the host: the first maximum flow, S_r / T_r, the
 * balance test, piercing and the incremental augmentation (Section 7; the
 * paper runs the FlowCutter problems of a round concurrently, Section 5,
 * "Parallel Scheduling").  Every decision is the one hfp_flowcutter takes, so
 * each task's outcome equals a hfp_flowcutter call on that network.
 * Networks must come fresh from hfp_build_flow_network (no flow computed),
 * belong to ctx and be distinct.  Per task: status receives HFP_OK,
 * HFP_NO_BALANCED_CUT, HFP_ABORTED_WORSE or an error code; final_side /
 * pierce_side / pierce_node (host, may be NULL) as in hfp_flowcutter.  The
 * call returns the first task error other than those two outcomes, or
 * HFP_ERR_BUFFER_TOO_SMALL when a piercing record did not fit.  Bulk
 * piercing and the most balanced cut are not supported here (a task asking
 * for them gives HFP_ERR_INVALID). */
typedef struct {
  hfp_net* net;
  hfp_fc_params params;
  uint8_t* final_side;     /* n_region */
  int32_t* pierce_side;    /* pierce_cap */
  int32_t* pierce_node;    /* pierce_cap */
  int32_t pierce_cap;
  hfp_status status;       /* out */
  hfp_fc_result result;    /* out */
} hfp_fc_task;

hfp_status hfp_flowcutter_batch(hfp_ctx* ctx, hfp_fc_task* tasks, int32_t n, int32_t group_ctas);

/* Profile of the batched launches (hfp_flowcutter_batch and the batched
 * k-way rounds) since the last reset, summed over their networks: the
 * device time (globaltimer, measured by each group's first CTA) a group
 * spent in each engine state, and the number of phases, for states
 * 0 .. n_states - 1 (at most 24; the numbering of hfp_net_get_trace, plus
 * 10 saturation of a new source, 11 piercing-key maximum with its holder
 * (12 unused), 13 / 14 marking S / T, 15 / 16 S_r / T_r grown from one node, 17 / 18
 * queue-driven global relabel seed / search, 19 one-phase round, 20 flush
 * of its pushes; phases run by one CTA count as 9), and the summed input
 * sizes of those phases, light_in / heavy_in (nodes of at most / more than
 * 16 arc groups in the frontier, the list being applied, or the
 * breadth-first-search level; for state 11 light_in counts the nets whose
 * pins the selection walked; 0 for other states).  reset != 0 zeroes the
 * sums after copying.  Host memory; any pointer may be NULL.  No paper
 * counterpart. */
hfp_status hfp_ctx_batch_profile(hfp_ctx* ctx, uint64_t* state_ns, uint64_t* state_cnt,
                                 uint64_t* light_in, uint64_t* heavy_in, int32_t n_states,
                                 int32_t reset);

/* Layout of the context's last batched FlowCutter launch: the number of
 * groups, CTAs per group, and 1 when the groups were thread-block clusters
 * (0: one cooperative launch).  Host pointers, any may be NULL.  No paper
 * counterpart. */
hfp_status hfp_ctx_last_batch_layout(hfp_ctx* ctx, int32_t* groups, int32_t* group_ctas,
                                     int32_t* cluster);

/* Failure path of the device waits: one launch of 2 CTAs whose barrier
 * (barrier 0: the engine's grid barrier; 1: a batched group's barrier in
 * global memory; 2: a cluster barrier in distributed shared memory, the two
 * CTAs then forming one thread-block cluster) waits for one arrival more than
 * the launch has CTAs, so only the context's wait_timeout_ms ends it.
 * Returns HFP_ERR_ITER_LIMIT when the wait ran out as designed, with
 * *waited_ms (host, may be NULL) the launch's device time; HFP_OK would mean
 * a barrier completed without all its arrivals.  The context stays usable.
 * HFP_ERR_INVALID for barrier outside 0..2.  No paper counterpart. */
hfp_status hfp_ctx_wait_selftest(hfp_ctx* ctx, int32_t barrier, float* waited_ms);

/* --- k-way refinement (Section 4, Algorithm 1; Sections 5 and 6) ---------
 * A device-resident hypergraph (with its vertex -> nets incidence) for
 * refining k-way partitions block pair by block pair.  Partitions are int32
 * block ids in [0, k) in DEVICE memory, k <= 64. */
typedef struct hfp_hgraph hfp_hgraph;

typedef struct {
  int32_t eps_pct;        /* balance: L = floor((100 + eps_pct) * ceil(c(V) / k) / 100) [3] */
  int32_t alpha_eps_pct;  /* region bound: 100 * alpha * eps [48: alpha = 16, eps = 0.03] */
  int32_t delta;          /* region vertices are at most delta hops from the pair's cut [2] */
  uint32_t seed;          /* third piercing key of FlowCutter */
} hfp_refine_params;

typedef struct {
  int32_t bi, bj;          /* the block pair */
  int32_t status;          /* HFP_OK, HFP_NO_BALANCED_CUT or HFP_ABORTED_WORSE */
  int32_t region_size;
  int64_t pins;            /* Lawler-network pins of the pair's flow network */
  int64_t original_cut;    /* weight of the network's nets cut by the input partition */
  int64_t flow;            /* final flow = cut weight of FlowCutter's bipartition */
  int64_t delta_exp;       /* original_cut - flow (Algorithm 1: Delta_exp) */
  int32_t n_moves;         /* region vertices that change block */
  int32_t iterations;      /* FlowCutter augmentations */
  int32_t applied;         /* hfp_refine_round: 1 if the moves were kept */
  int32_t valid_moves;     /* hfp_refine_round: moves that were not stale */
  int64_t gain;            /* hfp_refine_round: actual reduction of (lambda - 1) */
  int32_t device_us;       /* batched round: device time of the pair's FlowCutter */
  int32_t group_ctas;      /* batched round: CTAs of the group that solved it */
} hfp_pair_result;

typedef struct {
  int64_t connectivity_before, connectivity_after;  /* (lambda - 1), Section 2 */
  int64_t gain;            /* connectivity_before - connectivity_after */
  int64_t moves_applied;
  int32_t pairs;           /* pairs refined */
  int32_t pairs_improved;  /* pairs with Delta_exp > 0 */
  int32_t pairs_applied;   /* move sets kept */
  int32_t pairs_skipped;   /* pairs below min_score */
  /* host wall-clock milliseconds of the round's parts: quotient graph and
   * pair list, regions + networks (+ FlowCutter in hfp_refine_round), the
   * batched FlowCutter launch (0 in hfp_refine_round), move extraction,
   * apply step */
  float ms_pairs, ms_prepare, ms_flow, ms_finish, ms_apply;
  int32_t pad;
} hfp_round_stats;

/* Uploads H (in `mem` memory) and builds its vertex -> nets incidence. */
hfp_status hfp_hgraph_create(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                             hfp_hgraph** out);
void hfp_hgraph_destroy(hfp_hgraph* hg);
/* (lambda - 1)(part) = sum over nets of (lambda(e) - 1) w(e) (Section 2). */
hfp_status hfp_connectivity(hfp_hgraph* hg, const int32_t* part, int32_t k, int64_t* value);

/* One block pair of Algorithm 1 against partition `part` (device): grow the
 * region B (Section 6: breadth-first search inside each block from its pins
 * of the pair's cut nets, up to delta hops, vertices taken level by level in
 * ascending id while the block's share stays within
 * max(0, floor((100 + alpha_eps_pct) * ceil((c(Vi)+c(Vj))/2) / 100) - c(Vj))),
 * build its flow network with those distances, run FlowCutter with the k-way
 * bound L and the original pair cut as flow bound, and report the moves
 * (vertex, from, to) in ascending vertex order (host buffer of 3 * cap
 * int32) and Delta_exp = original cut - final flow.  A FlowCutter that finds
 * no balanced cut or exceeds the bound gives res->status != HFP_OK and no
 * moves; the call itself still returns HFP_OK.  k <= 64 (block masks of the
 * nets), else HFP_ERR_INVALID. */
hfp_status hfp_refine_block_pair(hfp_hgraph* hg, const int32_t* part, int32_t k, int32_t bi,
                                 int32_t bj, const hfp_refine_params* params, int32_t* moves,
                                 int32_t cap, hfp_pair_result* res);

/* One synchronous round of Algorithm 1 on `part` (device, updated): every
 * pair of adjacent blocks (quotient graph, Section 5) is refined against the
 * same partition; pairs with pair_scores[i * k + j] < min_score are skipped
 * (pair_scores host k * k, or NULL).  The move sets with Delta_exp >= 0 are
 * applied in descending Delta_exp (ties ascending (i, j)) by the rules of
 * Section 5, "Apply Moves": stale moves are dropped, a set is skipped if a
 * block that gains weight would exceed L, and reverted if its actual gain
 * is negative.  pairs (host, cap entries, may be NULL) receives the per-pair
 * results in ascending (i, j). */
hfp_status hfp_refine_round(hfp_hgraph* hg, int32_t* part, int32_t k,
                            const hfp_refine_params* params, const float* pair_scores,
                            float min_score, hfp_round_stats* stats, hfp_pair_result* pairs,
                            int32_t cap, int32_t* n_pairs);

/* hfp_refine_round with all FlowCutter problems of the round in ONE batched
 * launch (hfp_flowcutter_batch): regions and networks are built first, the
 * batch runs, then moves are extracted and applied exactly as in
 * hfp_refine_round, so the outcome is identical.  group_ctas: CTAs per
 * problem (<= 0: the value picked by hfp_autotune_round, else one group per
 * problem as far as the grid allows).  flowcutter_ms (host, may be NULL):
 * device time of the batched launch. */
hfp_status hfp_refine_round_batched(hfp_hgraph* hg, int32_t* part, int32_t k,
                                    const hfp_refine_params* params, const float* pair_scores,
                                    float min_score, int32_t group_ctas, hfp_round_stats* stats,
                                    hfp_pair_result* pairs, int32_t cap, int32_t* n_pairs,
                                    float* flowcutter_ms);

/* Autotuner of the batched round's tiling: builds the round's networks for
 * `part` (unchanged) once per candidate group size (CTAs per problem),
 * times the batched FlowCutter launch for each (ms[c], host, may be NULL),
 * and keeps the fastest in hg for hfp_refine_round_batched (*best). */
/* Autotuner of the batched round's engine knobs (beyond the group size):
 * with group_ctas CTAs per problem (<= 0: the autotuned or default size) it
 * builds the round's networks for `part` (unchanged) once per try and times
 * the batched launch for, in turn, gr_work_x100 in {100, 200, 400},
 * stall_rounds_pierce in {0 (adaptive), 30, 100}, (tail_enter, tail_exit) in
 * {(64, 192), (16, 64), (256, 768)} and batch_fused_rounds in {1, 0}, each
 * knob from the best setting found so far (starting from the context's
 * batched-launch knobs; gr_work_x100 and stall_rounds_pierce stand for their
 * batch_ forms here and in *chosen).  ms[cap] (host, may be NULL when
 * cap is 0) receives the launch times in that order, *n_tried their count;
 * the fastest setting is kept in hg for its batched rounds and returned in
 * *chosen (the context's tuning with those knobs; may be NULL).  Single flows
 * and other hypergraphs keep the context's knobs.  No paper counterpart. */
hfp_status hfp_autotune_round_engine(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                     const hfp_refine_params* params, int32_t group_ctas,
                                     float* ms, int32_t cap, int32_t* n_tried,
                                     hfp_tuning* chosen);
hfp_status hfp_autotune_round(hfp_hgraph* hg, const int32_t* part, int32_t k,
                              const hfp_refine_params* params, const int32_t* candidates,
                              int32_t n_candidates, float* ms, int32_t* best);

/* --- one round in three calls ---------------------------------------------
 * Algorithm 1 refines all block pairs of a round against the same partition
 * and only then applies their move sets (Section 5, "Parallel Scheduling",
 * "Apply Moves").  The pairs are therefore independent problems that several
 * processes (one GPU each) can share; the apply step needs every pair's
 * moves.  These calls expose the three stages: the pair list, the refinement
 * of any subset of it, and the apply step over move sets gathered from all
 * processes.  Refining every pair in one call and applying gives exactly
 * hfp_refine_round_batched's outcome, whatever the split. */

/* Edges of the quotient graph of `part` (device; Section 5, "Quotient Graph
 * Construction"): every pair i < j of blocks with a net in both, ascending
 * (i, j), without pairs whose pair_scores[i*k + j] (host, k*k; NULL: none)
 * is below min_score.  pairs: host int32[cap][2]; pair_nets (host, may be
 * NULL): int64[cap], the number of nets in both blocks (a size estimate);
 * *n_pairs: the count (HFP_ERR_BUFFER_TOO_SMALL when above cap, *n_pairs
 * still set); *connectivity (may be NULL): (lambda - 1)(part). */
hfp_status hfp_round_pairs(hfp_hgraph* hg, const int32_t* part, int32_t k,
                           const float* pair_scores, float min_score, int32_t* pairs,
                           int64_t* pair_nets, int32_t cap, int32_t* n_pairs,
                           int64_t* connectivity);

/* Refines the n given pairs (host int32[n][2], 0 <= i < j < k, no repeats)
 * against `part` (device, unchanged), exactly as hfp_refine_round_batched
 * does (region, network, FlowCutter in one batched launch with group_ctas
 * CTAs per problem, moves), without applying anything.  results[t] (host)
 * is pair t's outcome; its moves (vertex, from block, to block) go to host
 * moves[3 * move_off[t]] .. moves[3 * move_off[t + 1] - 1], move_off being
 * host int64[n + 1].  HFP_ERR_BUFFER_TOO_SMALL when the moves exceed
 * move_cap triples (move_off is filled: move_off[n] is the need).
 * flowcutter_ms (may be NULL): device time of the batched launch. */
hfp_status hfp_refine_pairs_batched(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                    const hfp_refine_params* params, const int32_t* pairs,
                                    int32_t n, int32_t group_ctas, hfp_pair_result* results,
                                    int32_t* moves, int64_t move_cap, int64_t* move_off,
                                    float* flowcutter_ms);

/* The apply step of a round (Section 5, "Apply Moves") on n pair results
 * and their moves (host, the layout of hfp_refine_pairs_batched, in any
 * order of the pairs): the move sets of pairs with status HFP_OK,
 * Delta_exp >= 0 and at least one move, in descending Delta_exp with ties in
 * ascending (bi, bj), each checked for stale moves and balance and reverted
 * when its actual gain is negative.  part (device) is updated; results[t]
 * receives applied, valid_moves and gain; stats the round's totals
 * (connectivity before and after, gain, pairs, moves applied, ms_apply).
 * HFP_ERR_INVALID for a result whose move count disagrees with move_off or
 * a move that is not between the pair's two blocks. */
hfp_status hfp_apply_moves(hfp_hgraph* hg, int32_t* part, int32_t k,
                           const hfp_refine_params* params, hfp_pair_result* results,
                           const int32_t* moves, const int64_t* move_off, int32_t n,
                           hfp_round_stats* stats);

/* --- learned block-pair scheduler ----------------------------------------
 * The paper has no learned component: its rounds refine every edge of the
 * quotient graph (Section 5, "Quotient Graph Construction" and "Parallel
 * Scheduling").  These calls score the edges with a multilayer perceptron
 * 16 -> 64 -> 64 -> 1 (ReLU, sigmoid output) so that hfp_refine_round can
 * skip pairs whose score is below a threshold (its pair_scores argument).
 * Weights and the inputs of the two matrix products are rounded to bfloat16
 * (nearest even); products accumulate in fp32; the last layer is an fp32 dot
 * product with bf16 weights.  Parameters are one fp32 array of
 * HFP_MLP_PARAMS values: W1[64][16], b1[64], W2[64][64], b2[64], w3[64],
 * b3 (row-major, W[out][in]).  All pointers except the noted host ones are
 * device pointers. */
#define HFP_MLP_FEATURES 16
#define HFP_MLP_HIDDEN 64
#define HFP_MLP_PARAMS 5313

/* Features of every block pair i < j joined by a net (row-major pair
 * order), from counts over those nets: with "nets2" the joining nets whose
 * blocks are exactly {i, j}, L = floor((100 + eps_pct) * ceil(c(V) / k) / 100):
 *   0 log1p(nets)  1 log1p(weight)  2 log1p(pins)  3 log1p(largest net)
 *   4 log1p(nets2) 5 log1p(weight2) 6 weight2 / weight  7 log1p(pins2)
 *   8 c(Vi) / L    9 c(Vj) / L      10 (c(Vi) + c(Vj)) / (2 L)
 *   11 log1p(pins / nets)  12 log1p(max(prev, 0))  13 prev >= 0 ? 1 : 0
 *   14 log2(k) / 6  15 weight * P / (total weight of the P pairs)
 * prev_gain: host int64 k * k, gain of pair (i, j) in the previous round and
 * -1 where it was not refined, or NULL.  features: cap x 16 floats; pairs:
 * cap x 2 int32 (i, j); *n_pairs (host) = P; HFP_ERR_BUFFER_TOO_SMALL if
 * P > cap.  k in [2, 64].  Synchronises the context stream. */
hfp_status hfp_pair_features(hfp_hgraph* hg, const int32_t* part, int32_t k, int32_t eps_pct,
                             const int64_t* prev_gain, float* features, int32_t* pairs,
                             int32_t cap, int32_t* n_pairs);

/* scores[r] = sigmoid(MLP(x[r])) for rows x[rows][16]. */
hfp_status hfp_mlp_forward(hfp_ctx* ctx, const float* params, const float* x, int32_t rows,
                           float* scores);

/* Gradient (device, HFP_MLP_PARAMS floats) of the mean binary cross-entropy
 * of the logits against labels y[rows] (0 or 1); rounding to bf16 passes
 * the gradient straight through.  *loss (host, may be NULL) = the mean loss. */
hfp_status hfp_mlp_grad(hfp_ctx* ctx, const float* params, const float* x, const float* y,
                        int32_t rows, float* grad, float* loss);

typedef struct {
  float lr;
  float eps;
  double beta1;
  double beta2;
} hfp_adam_params;

/* `steps` full-batch Adam steps (Kingma and Ba, 2015) on params with moment
 * arrays adam_m, adam_v (HFP_MLP_PARAMS floats each, zero before the first
 * step) and the device step counter *step (0 before the first step;
 * incremented per step).  One step is a forward/backward launch and a
 * reduce/update launch, captured once as a CUDA graph and replayed.
 * losses (device, loss_cap floats, may be NULL) receives the mean loss of
 * the i-th step of this call at index i - 1 while i <= loss_cap.  Synchronises the context
 * stream. */
hfp_status hfp_mlp_train(hfp_ctx* ctx, float* params, float* adam_m, float* adam_v,
                         int32_t* step, const float* x, const float* y, int32_t rows,
                         int32_t steps, const hfp_adam_params* opt, float* losses,
                         int32_t loss_cap);

/* hfp_pair_features + hfp_mlp_forward, scattered into a host k * k table
 * (scores[i * k + j] for i < j joined by a net, -1 elsewhere) in the form
 * hfp_refine_round takes. */
hfp_status hfp_pair_scores(hfp_hgraph* hg, const int32_t* part, int32_t k, int32_t eps_pct,
                           const int64_t* prev_gain, const float* params, float* scores);

/* --- allocation-free max flow ---------------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory where they need a flow: a plug-in bound
 * to a host application's fixed device-memory budget or allocator, or a
 * loop in which allocation is forbidden (cudaMalloc may synchronise the
 * device or fail under memory pressure).  It computes what hfp_max_flow +
 * hfp_min_cut_source_side compute for the flow problem {s} -> {t} of a
 * network, with the same engine kernel, but keeps all working state in one
 * fixed static device array of 24 MiB (library-wide, held by every GPU that
 * loads the library until the process exits).  It calls no cudaMalloc /
 * cudaFree and no allocating library routine.
 *   net: the flow network in device memory, in the layout hfp_net_export
 *        writes (hypernode 0 = s, 1 = t).  It fits when
 *        47*L + 20*p + 4*m + 5 KiB <= 24 MiB (L = n_nodes + 2*m_nets Lawler
 *        nodes, p pins, m nets; e.g. L = 262,144 with p = 524,288);
 *        larger networks are rejected with HFP_ERR_INVALID, and so are views
 *        whose offsets or ids are out of range or whose incidence lists do
 *        not name every pin slot of the node exactly once.
 *   flow_value, source_weight: host pointers (may be NULL);
 *   in_source_lawler[L]: device pointer (may be NULL), 1 for nodes of S_r.
 * The first call on a device looks up the array's device address (with that
 * device current).  Every call shares the array and clears what it uses;
 * calls that overlap on the GPU race, so serialise them.  The call
 * synchronises `stream` and reads status words back to the host, so it
 * cannot run inside a CUDA stream capture. */
typedef struct {
  int32_t n_nodes;
  int32_t m_nets;
  int64_t p_pins;
  const uint32_t* net_off;   /* m_nets + 1 */
  const int32_t* pins;       /* p_pins */
  const int32_t* net_w;      /* m_nets */
  const uint32_t* node_off;  /* n_nodes + 1 */
  const int32_t* inc_slot;   /* p_pins: pin slots of each hypernode */
  const int32_t* node_w;     /* n_nodes */
} hfp_flow_network_view;

hfp_status hfp_max_flow_noalloc(int device, void* stream, const hfp_flow_network_view* net,
                                int64_t* flow_value, uint8_t* in_source_lawler,
                                int64_t* source_weight);

#ifdef __cplusplus
}
#endif

#endif /* HFP_H */
