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
};

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
  int pad;
  unsigned long long rounds, grs, gr_levels, work, stall, flow, flow_ref;
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
  unsigned int pad;
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
};

}  // namespace hfp
