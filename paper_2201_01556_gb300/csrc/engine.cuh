// Flow engine: state shared by the persistent push-relabel / BFS kernel and
// the host.  See engine.cu for the algorithm.
#pragma once
#include "common.cuh"

namespace hfp {

// Engine states (Sched::state).  The grid walks through them; each change
// happens in the serial section of a grid barrier.
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
};

// list ids in NetDev::list
enum ListId : int { L_FRONT = 0, L_NEXT = 1, L_RELAB = 2, L_BFS = 3 };

struct Sched {
  int state;
  int lp;                 // current labels live in lab[lp]
  unsigned int fcnt;      // frontier size of this round
  unsigned int ncnt;      // next-list size (phase B input)
  unsigned int rcnt;      // relabeled-last-round list size (fix-ups in phase A)
  unsigned int bfs_begin, bfs_end;  // current BFS level = list[L_BFS][begin, end)
  int level;
  unsigned int epoch;     // stamp epoch of this round / BFS
  int final_gr;           // the running global relabel follows termination
  int after_gr_exit;      // exit after the running global relabel
  int stop_after_sr;      // exit after the source-side BFS
};

struct Params {
  unsigned long long timeout_ns;     // bound on every grid-barrier wait
  unsigned long long max_rounds;     // discharge round budget
  unsigned long long gr_work;        // arcs scanned between global relabels
  unsigned long long stall_rounds;   // rounds without flow change ...
  unsigned int stall_nodes;          // ... each with fewer active nodes
};

struct EngineCtl {
  Ctl c;
  Sched s;
  unsigned int cnt[4];               // append counters of the lists
  unsigned long long round_flow_ref;  // flow value when the stall window opened
};

}  // namespace hfp
