// Flow engine: state shared by the persistent push-relabel / BFS kernel and
// the host.  See engine.cu for the algorithm.
#pragma once
#include "common.cuh"

namespace hfp {

// Engine states.  All CTAs walk through them in lockstep; every CTA derives
// the next state itself from the counters of the phase that just ended.
enum EngineState : int {
  ST_DONE = 0,
  ST_ROUND_A = 1,   // discharge the frontier (pushes only)
  ST_ROUND_B = 2,   // apply excess deltas, relabel, build the next frontier
  ST_GR_INIT = 3,   // global relabel: reset labels, seed sinks
  ST_GR_LEVEL = 4,  // global relabel: one reverse-BFS level
  ST_SR_INIT = 5,   // source-side cut: seed S and the non-sink excess nodes
  ST_SR_LEVEL = 6,  // source-side cut: one forward-BFS level
  ST_DIST_INIT = 7, // distance from the cut: seed the distance-1 vertices
  ST_DIST_LEVEL = 8,  // distance from the cut: one BFS level inside the region
  ST_TAIL = 9,      // rounds run by CTA 0 alone while the frontier is small
  // batched FlowCutter (fc_batch_kernel): the steps of Algorithm 2 around the flow
  ST_FC_SAT = 10,     // saturate the arcs out of a new source hypernode
  ST_FC_SEL = 11,     // largest piercing key over the candidates, and its holder
  ST_FC_FIND = 12,    // (unused: the holder comes with the key)
  ST_FC_MARK_S = 13,  // S <- S_r + pierced node
  ST_FC_MARK_T = 14,  // T <- T_r + pierced node, their excess joins the flow
  ST_SR_ADD = 15,   // source-side cut grown from one new source (S_r kept)
  ST_GR_ADD = 16,   // sink-side cut grown from one new sink (T_r and its labels kept)
  ST_GR_SEED = 17,  // asynchronous global relabel: the sinks enter the work queue
  ST_GR_RUN = 18,   // asynchronous global relabel: label-correcting search to the end
  ST_ROUND = 19,    // one-phase round: apply last round's pushes, discharge, relabel
  ST_FLUSH = 20,    // apply the pushes of the last one-phase round (before a relabel)
};

// Slots of per-state time accounting (states 0 .. ST_FLUSH).
constexpr int kStateSlots = 24;

// list ids in NetDev::list.  Each list array holds light nodes from the front
// and heavy nodes from the back (heavy entry i sits at NL - 1 - i); a node is
// in a list at most once, so the two never meet.
enum ListId : int { L_FRONT = 0, L_NEXT = 1, L_RELAB = 2, L_BFS = 3 };
// append counters
enum CntId : int { C_FRONT = 0, C_FRONTH = 1, C_NEXT = 2, C_NEXTH = 3, C_RELAB = 4, C_BFS = 5,
                   C_BFSH = 6, C_COUNT = 7 };

// Engine state as published between launches (and by CTA 0 after a tail).
struct Sched {
  int state;
  int lp;                 // current labels live in lab[lp]
  unsigned int fcnt, fcnth;  // frontier of the next round (light, heavy)
  unsigned int ncnt, ncnth;  // next list (phase B input; light, heavy)
  unsigned int rcnt;         // relabeled-last-round list size (fix-ups in phase A)
  unsigned int bfs_begin, bfs_end;    // current BFS level, light part
  unsigned int bfsh_begin, bfsh_end;  // current BFS level, heavy part
  int level;
  unsigned int epoch;     // stamp epoch of this round / BFS
  int after_gr_exit;      // exit after the running global relabel
  unsigned int phase;     // phase index (selects the counter slots)
  int seed;               // ST_SR_ADD / ST_GR_ADD: the node whose reach joins S_r / T_r
  unsigned int last_gr;   // levels of the last global relabel
  int gr_sync;            // this global relabel runs level by level (queue overflowed)
  int fsel;               // one-phase rounds: list holding the frontier (L_FRONT / L_NEXT)
  unsigned long long rounds, grs, gr_levels, work, stall, flow, flow_ref;
  unsigned long long gq_items, gq_overs;   // queue entries expanded, queue overflows
  unsigned gq_prev;       // queue slots written by the last asynchronous relabel
  unsigned gq_pad;
  // Seeds of the searches from the terminal sets: 0 seeds every sink (global
  // relabel) / every source (S_r); v + 1 seeds only the terminal v, the one
  // terminal that can have residual arcs to (from) the other nodes.  The
  // other terminals still get label 0 / join S_r, they are only not expanded.
  int gr_one, sr_one;
  long long wS, wT;
  int wS_set, wT_set;
};

struct Params {
  unsigned long long timeout_ns;     // bound on every grid-barrier wait
  unsigned long long max_rounds;     // discharge round budget
  unsigned long long gr_work;        // list entries processed between global relabels
  unsigned long long stall_rounds;   // rounds without flow change ...
  unsigned int stall_nodes;          // ... each with fewer active nodes
  unsigned int tail_enter;           // frontier size at or below which CTA 0 runs alone
  unsigned int tail_exit;            // frontier size above which the grid takes over
  unsigned int bfs_enter;            // BFS level size at or below which CTA 0 runs alone
  unsigned int bfs_exit;             // BFS level size above which the grid takes over
  unsigned int pierce_relabel;       // source piercing: start the flow with a global relabel
  unsigned int stall_rounds_pierce;  // stall_rounds of the flows after a piercing (0: adaptive)
  unsigned int stall_adapt;          // stall limit = levels of the last global relabel
  unsigned int async_gr;             // global relabels as one queue-driven search
  unsigned int gr_warps;             // warps per CTA that serve that search's queue
  unsigned int fused_rounds;         // one phase per discharge round (needs NetDev::delta1)
  unsigned int parpr_block;          // one-phase rounds relabel by ParPR-Block (needs NetDev::blk)
};

struct EngineCtl {
  Ctl c;
  Sched s;
  unsigned int cnt[2];               // frontier appends outside the engine (k_saturate)
  unsigned int cnt3[C_COUNT][3];     // per-phase append counters, slot = phase % 3
  unsigned int gr_act[2];            // active nodes found by the running global relabel
  unsigned int bar_count;            // count-up grid barrier (reset per launch)
  unsigned long long flow3[3];       // flow into sinks per phase slot
  long long w3[3];                   // hypernode weight reached per phase slot
  unsigned long long key3[3];        // batched FlowCutter: best piercing key per slot
  int node3[3];                      // batched FlowCutter: node holding it per slot
  int pad3;
  // work queue of the asynchronous global relabel, one counter per 128-byte
  // line (entries handed out, entries written, entries finished)
  alignas(128) unsigned gq_head;
  alignas(128) unsigned gq_tail;
  alignas(128) unsigned gq_done;
  unsigned gq_over;                  // an entry did not fit: redo level by level
  unsigned gq_maxd;                  // largest label set by the search
};

// One flow problem of a batched FlowCutter launch (Section 7, Algorithm 2):
// the network, its control block, the FlowCutter parameters and, written by
// the kernel, the outcome.
struct FcJob {
  NetDev N;
  EngineCtl* E;
  long long total_w;          // c(V) of the network, terminals included
  long long max_w;            // balance bound L
  long long flow_bound;       // abort above this flow (-1: none)
  unsigned long long gr_work; // global-relabel work threshold of this network
  int32_t* pierce_node;       // piercing record (pierce_cap entries, may be null)
  int8_t* pierce_side;
  uint32_t seed;
  int32_t max_it;
  int32_t dist_ready;         // distances given at construction
  int32_t pierce_cap;
  // outcome
  int32_t status;             // 0, or an hfp_status (<0), or 100 + device error code
  int32_t iterations;
  int32_t n_pierced;
  int32_t result_side;        // 0: S_r side, 1: T_r side
  long long flow;
  long long source_weight;
  unsigned long long device_ns;  // globaltimer time of the job in its group
  int32_t group_ctas;            // CTAs of that group
  int32_t pad;
  // group time per engine state (phases run by one CTA count as ST_TAIL)
  unsigned long long st_ns[kStateSlots];
  unsigned st_cnt[kStateSlots];
  unsigned long long st_lin[kStateSlots], st_hin[kStateSlots];   // light / heavy inputs
};

// Work queue and per-group barriers of a batched launch.
constexpr int kMaxGroups = 1024;
constexpr int kMaxBatchCtas = 1024;
struct BatchCtl {
  unsigned next;              // next job to hand out
  int err;                    // a group barrier timed out
  unsigned gbar[kMaxGroups];  // count-up barrier per group
  unsigned gjob[kMaxGroups];  // job handed to each group
  // per CTA: its largest piercing key and the node holding it (ST_FC_SEL)
  unsigned long long sel_key[kMaxBatchCtas];
  int sel_node[kMaxBatchCtas];
};

}  // namespace hfp
