// Persistent flow engine: synchronous push-relabel on the Lawler expansion,
// simulated directly on the flow hypergraph, with global relabeling and the
// residual BFS of the source-side cut.  One cooperative launch runs the whole
// loop.  Every CTA derives the next state itself from the counters of the
// phase that just ended (the counters rotate through three slots, so none is
// reset while it is read or written); small frontiers are discharged by CTA 0
// alone with block barriers while the other CTAs wait.
//
// Light nodes (at most kLightItems arc groups) are handled by teams of kTeam
// lanes, which place their pushes by a team scan of residual capacities.
// Heavy nodes (large nets, s, t, high-degree vertices) get a whole CTA, which
// scans blockDim.x arc groups per step and places pushes by a block scan.
//
// Method (Section 8 of the paper, "Parallel Maximum Flow Algorithm"):
//  - rounds discharge all active nodes in parallel against the labels and
//    excesses of the previous round; excess deltas are summed atomically and
//    applied afterwards (Section 8.1);
//  - the hypergraph is not expanded: three discharge routines handle
//    hypernodes, in-nodes and out-nodes (Section 8.3, "Hypergraph
//    Implementation");
//  - arcs (u, e_in) are capped at w(e) during the preflow (Section 8.3,
//    "Restricting Capacities");
//  - global relabeling is a reverse BFS from the sinks; it also collects the
//    active nodes and yields the sink-side cut T_r (Sections 8.1, 8.2, 8.3);
//  - sinks never enter the frontier; pushes into a sink add to the flow
//    value directly (Section 8.3, "Flow Value");
//  - the source-side cut is a forward residual BFS seeded with the sources
//    and every non-sink excess node, treating (u, e_in) as uncapped
//    (Section 8.4, "Source-Side Cut"; Section 8.3, last paragraph of
//    "Restricting Capacities").
//
// Difference from the paper's round.  Two round forms are built, and both
// keep every label valid, so the push-relabel conflict of Section 8.2 cannot
// occur and no winning criterion is needed:
//  - two-phase rounds (ROUND_A / ROUND_B): pushes use only the old labels,
//    and a node relabels (against the old labels of its neighbours, read from
//    the other buffer of a double-buffered label array) only after every push
//    of the round has landed;
//  - one-phase rounds (ROUND / FLUSH, the default of single flows): a node
//    applies the pushes it received in the previous round, discharges and
//    relabels itself at once with the capped rule explained at phase_round.
// Global relabeling is either level-synchronous (one grid phase per BFS
// level) or one queue-driven label-correcting search (GR_SEED / GR_RUN).
// Runs are deterministic: excess moves by integer atomics only, and the
// queue-driven search ends at the exact BFS distances the level-synchronous
// one computes.  The two round forms reach the same flow value and cuts
// (both unique) in different numbers of rounds.
#include <climits>

#include "kernels.cuh"

namespace hfp {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kTeam = 8;   // lanes per light node

struct Acc {
  long long w;                 // hypernode weight found in this phase
  unsigned long long hyper, net, nodes, pushes;
};

// Iteration space of a phase: the whole grid, or CTA 0 alone in the tail.
// Light nodes go to 8-lane teams over all warps; heavy nodes to whole CTAs
// (block b takes heavy nodes b, b + nblocks, ...).
struct Team {
  unsigned gwarp, nwarps, tid, nth, block, nblocks;
};

// Append counters and accumulators of the current phase: slot phase % 3 of
// the control block in grid phases, shared memory in CTA-alone phases.
struct Slot {
  unsigned* c[C_COUNT];
  unsigned long long* flow;
  unsigned* act[2];            // active nodes found by the running global relabel
};

// Counters of CTA-alone phases (shared memory of the CTA running them).
struct SoloSh {
  unsigned c[C_COUNT];
  unsigned act[2];
  unsigned long long flow;
  int stay;
};

__device__ __forceinline__ int32_t* lab_cur(const NetDev& N, int lp) { return lp ? N.lab1 : N.lab0; }

__device__ __forceinline__ unsigned warp_max_u(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(FULL, v, o));
  return v;
}

// Warp-aggregated append to a split list: light values at
// list[base_l + i], heavy values at list[NL - 1 - (base_h + i)].  All 32
// lanes must call it together.
__device__ __forceinline__ void append_split(bool want, int32_t value, bool heavy, int32_t* list,
                                             unsigned* cl, unsigned* ch, unsigned base_l,
                                             unsigned base_h, int NL) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const unsigned ml = __ballot_sync(FULL, want && !heavy);
  const unsigned mh = __ballot_sync(FULL, want && heavy);
  if (ml) {
    const int leader = __ffs(ml) - 1;
    unsigned pos = 0;
    if ((int)lane == leader) pos = atomicAdd(cl, (unsigned)__popc(ml));
    pos = __shfl_sync(FULL, pos, leader);
    if (want && !heavy) list[base_l + pos + __popc(ml & lt)] = value;
  }
  if (mh) {
    const int leader = __ffs(mh) - 1;
    unsigned pos = 0;
    if ((int)lane == leader) pos = atomicAdd(ch, (unsigned)__popc(mh));
    pos = __shfl_sync(FULL, pos, leader);
    if (want && heavy) list[NL - 1 - (base_h + pos + __popc(mh & lt))] = value;
  }
}

// append_split for two values per lane (value 1 before value 2 of the same
// lane): one ballot pair and at most two atomics per warp.
__device__ __forceinline__ void append_split2(bool w1, int32_t v1, bool h1, bool w2, int32_t v2,
                                              bool h2, int32_t* list, unsigned* cl,
                                              unsigned* ch, unsigned base_l, unsigned base_h,
                                              int NL) {
  const unsigned lane = lane_id();
  const unsigned lt = (1u << lane) - 1u;
  const unsigned l1 = __ballot_sync(FULL, w1 && !h1), l2 = __ballot_sync(FULL, w2 && !h2);
  const unsigned g1 = __ballot_sync(FULL, w1 && h1), g2 = __ballot_sync(FULL, w2 && h2);
  const unsigned nl = __popc(l1) + __popc(l2), nh = __popc(g1) + __popc(g2);
  if (nl + nh == 0) return;
  unsigned pl = 0, ph = 0;
  if (lane == 0) {
    if (nl) pl = atomicAdd(cl, nl);
    if (nh) ph = atomicAdd(ch, nh);
  }
  pl = __shfl_sync(FULL, pl, 0);
  ph = __shfl_sync(FULL, ph, 0);
  unsigned o = pl + __popc(l1 & lt) + __popc(l2 & lt);
  if (w1 && !h1) list[base_l + o++] = v1;
  if (w2 && !h2) list[base_l + o] = v2;
  o = ph + __popc(g1 & lt) + __popc(g2 & lt);
  if (w1 && h1) list[NL - 1 - (base_h + o++)] = v1;
  if (w2 && h2) list[NL - 1 - (base_h + o)] = v2;
}

__device__ __forceinline__ void append_plain(bool want, int32_t value, int32_t* list,
                                             unsigned* cnt, unsigned base) {
  const unsigned m = __ballot_sync(FULL, want);
  if (!m) return;
  const unsigned lane = lane_id();
  const int leader = __ffs(m) - 1;
  unsigned pos = 0;
  if ((int)lane == leader) pos = atomicAdd(cnt, (unsigned)__popc(m));
  pos = __shfl_sync(FULL, pos, leader);
  if (want) list[base + pos + __popc(m & ((1u << lane) - 1u))] = value;
}

// Arc-group layout of node x: kind 0 hypernode (groups = incidences), kind 1
// in-node, kind 2 out-node (group 0 = bridge, group k = pin slot beg + k - 1).
struct NodeArcs {
  int kind, e;
  unsigned beg, items;
};

__device__ __forceinline__ NodeArcs node_arcs(const NetDev& N, int x) {
  NodeArcs r;
  const int nh = N.n_nodes, m = N.m_nets;
  if (x < nh) {
    r.kind = 0;
    r.e = 0;
    r.beg = N.node_off[x];
    r.items = N.node_off[x + 1] - r.beg;
  } else {
    r.kind = x < nh + m ? 1 : 2;
    r.e = r.kind == 1 ? x - nh : x - nh - m;
    r.beg = N.net_off[r.e];
    r.items = 1 + (N.net_off[r.e + 1] - r.beg);
  }
  return r;
}

// The light nodes nodes[0 .. count) (count <= 32) of a breadth-first level
// by one warp: every lane loads one node, and the warp walks the
// concatenated arc groups of the 32 nodes, 64 per step, so that a step costs
// one chain of dependent loads for up to 64 arc groups of different nodes
// (a team of lanes per node would wait once per node).  fn2(A, B) is called
// by every lane of the warp with two arc groups, positions q and q + 32 of
// the walk (k == kNoArc: none), and issues the loads of both before it waits
// on either; w and fb are the net's weight and bridge flow for net nodes.
constexpr unsigned kNoArc = 0xffffffffu;

struct WalkArc {
  NodeArcs g;
  unsigned k;
  int w, fb;
};

template <class Fn2>
__device__ __forceinline__ void warp_walk_arcs(const NetDev& N, const int32_t* nodes,
                                               unsigned count, unsigned lane, Fn2 fn2) {
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  if (lane < count) {
    g = node_arcs(N, nodes[lane]);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
  }
  unsigned incl = g.items;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const unsigned total = __shfl_sync(FULL, incl, 31);
  const unsigned excl = incl - g.items;
  // arc group at walk position q: its owner is the number of lanes whose
  // arcs end at or before q
  auto at = [&](unsigned q) {
    int own = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      const unsigned v = __shfl_sync(FULL, incl, own + step - 1);
      if (v <= q) own += step;
    }
    own = own < 31 ? own : 31;
    WalkArc r;
    r.g.kind = __shfl_sync(FULL, g.kind, own);
    r.g.e = __shfl_sync(FULL, g.e, own);
    r.g.beg = __shfl_sync(FULL, g.beg, own);
    r.g.items = __shfl_sync(FULL, g.items, own);
    r.w = __shfl_sync(FULL, w, own);
    r.fb = __shfl_sync(FULL, fb, own);
    const unsigned oex = __shfl_sync(FULL, excl, own);
    r.k = q < total ? q - oex : kNoArc;
    return r;
  };
  for (unsigned q0 = 0; q0 < total; q0 += 64) {
    const WalkArc A = at(q0 + lane);
    const WalkArc B = at(q0 + 32 + lane);
    fn2(A, B);
  }
}

// Node x (x < 0: idle team) by a team of kTeam lanes, kTeam arc groups per
// step; fn(g, k, w, fb) gets one arc group (k == kNoArc: none).
template <class Fn>
__device__ __forceinline__ void team_walk_arcs(const NetDev& N, int x, unsigned lane, Fn fn) {
  const unsigned tl = lane & (kTeam - 1);
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  if (x >= 0) {
    g = node_arcs(N, x);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
  }
  const unsigned steps = warp_max_u((g.items + kTeam - 1) / kTeam);
  for (unsigned c = 0; c < steps; c++) {
    const unsigned k = c * kTeam + tl;
    fn(g, k < g.items ? k : kNoArc, w, fb);
  }
}

// The light nodes nodes[0 .. count) of a breadth-first level over the warps
// of T: 32 per warp (warp_walk_arcs with fn2) when the level has more than
// kWalkMin nodes per warp, taken from the phase counter *grab (zero at the
// phase's start) so that the warps finish together; else one per team (fn),
// so that a small level still keeps every warp busy.
constexpr unsigned kWalkMin = 8;

template <class Fn, class Fn2>
__device__ __forceinline__ void level_light(const NetDev& N, const int32_t* nodes, unsigned count,
                                            const Team& T, unsigned lane, unsigned* grab, Fn fn,
                                            Fn2 fn2) {
  if (count > kWalkMin * T.nwarps) {
    for (;;) {
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(grab, 32u);
      base = __shfl_sync(FULL, base, 0);
      if (base >= count) break;
      warp_walk_arcs(N, nodes + base, min(32u, count - base), lane, fn2);
    }
  } else {
    constexpr unsigned TPW = 32 / kTeam;
    for (unsigned base = T.gwarp * TPW; base < count; base += T.nwarps * TPW) {
      const unsigned i = base + lane / kTeam;
      team_walk_arcs(N, i < count ? nodes[i] : -1, lane, fn);
    }
  }
}

// The heavy nodes of a breadth-first level (heavy entries hb .. hb + count
// of a split list), taken from the phase counter *grab (zero at the phase's
// start) count / CTAs at a time (at least 1, at most 32), so that a level's
// heavy nodes spread over all CTAs: warp 0 loads one node per lane, and the
// CTA walks the concatenated arc groups of those nodes 2 x blockDim.x per
// step, two per thread (fn2 as in warp_walk_arcs).  (A CTA per node would
// leave most threads idle for the typical heavy node of a few dozen arc
// groups and take the nodes one after another.)  Every thread of the CTA
// must call this.
struct HeavyStep {
  NodeArcs g[32];
  int w[32], fb[32];
  unsigned incl[32];
};

template <class Fn2>
__device__ __forceinline__ void block_walk_heavy(const NetDev& N, const int32_t* list, unsigned hb,
                                                 unsigned count, const Team& T, unsigned* grab,
                                                 Fn2 fn2) {
  __shared__ HeavyStep H;
  __shared__ unsigned h0_sh;
  const unsigned take = min(32u, max(1u, (count + T.nblocks - 1) / T.nblocks));
  for (;;) {
    // the next entries for this CTA, from the phase counter *grab
    if (threadIdx.x == 0) h0_sh = count ? atomicAdd(grab, take) : count;
    __syncthreads();
    const unsigned h0 = h0_sh;
    if (h0 >= count) break;
    if (threadIdx.x < 32) {
      const unsigned t = threadIdx.x;
      NodeArcs g{0, 0, 0, 0};
      int w = 0, fb = 0;
      if (t < take && h0 + t < count) {
        g = node_arcs(N, list[N.NL - 1 - (hb + h0 + t)]);
        if (g.kind) {
          w = N.net_w[g.e];
          fb = N.f_b[g.e];
        }
      }
      unsigned incl = g.items;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(FULL, incl, o);
        if ((int)t >= o) incl += v;
      }
      H.g[t] = g;
      H.w[t] = w;
      H.fb[t] = fb;
      H.incl[t] = incl;
    }
    __syncthreads();
    const unsigned total = H.incl[31];
    auto at = [&](unsigned q) {
      int own = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1)
        if (H.incl[own + step - 1] <= q) own += step;
      own = own < 31 ? own : 31;
      WalkArc r;
      r.g = H.g[own];
      r.k = q < total ? q - (H.incl[own] - r.g.items) : kNoArc;
      r.w = H.w[own];
      r.fb = H.fb[own];
      return r;
    };
    for (unsigned q0 = 0; q0 < total; q0 += 2 * blockDim.x) {
      const WalkArc A = at(q0 + threadIdx.x);
      const WalkArc B = at(q0 + blockDim.x + threadIdx.x);
      fn2(A, B);
    }
    __syncthreads();   // H is rewritten by the next step
  }
}

// ---------------------------------------------------------------------------
// Control: every CTA's thread 0 runs this after each barrier on its own copy
// of the state, with the counters of the phase that ended.  The decisions
// only depend on values that no CTA changes during the next phase, so all
// copies stay identical.
struct Snap {
  unsigned c[C_COUNT];
  unsigned act, acth;
  unsigned long long flow;
  long long w;
  unsigned long long key;
  int node;
  unsigned gq_over, gq_maxd;   // asynchronous global relabel: overflow, largest label
  unsigned gq_tail;            // ... and the entries it queued
};

// Rounds without flow change before a global relabel (Section 8.3, "Avoid
// Pushing Flow Back").  In adaptive mode (incremental flows after a
// piercing) the limit follows the cost of a relabel: as many rounds as the
// last one had levels, at least 8, at most kStallAdaptCap.
constexpr unsigned long long kStallAdaptCap = 200;

__device__ __forceinline__ unsigned long long stall_limit(const Sched& L, const Params& P) {
  if (!P.stall_adapt) return P.stall_rounds;
  unsigned long long s = L.last_gr < 8u ? 8u : L.last_gr;
  return s < kStallAdaptCap ? s : kStallAdaptCap;
}

__device__ void begin_gr(Sched& L) {
  L.grs++;
  L.state = ST_GR_INIT;
  L.wT = 0;
  L.wT_set = 1;
}

// The discharge round of this configuration: one phase, or push and
// relabel phases.
__device__ __forceinline__ int round_state(const Params& P) {
  return P.fused_rounds ? ST_ROUND : ST_ROUND_A;
}

// End of a global relabel with `levels` breadth-first levels: the active
// nodes it found form the frontier; labels are exact distances.
__device__ __forceinline__ void end_gr(Sched& L, const Snap& q, const Params& P, unsigned levels) {
  L.last_gr = levels;
  L.gr_sync = 0;
  L.fcnt = q.act;
  L.fcnth = q.acth;
  L.rcnt = 0;
  L.lp = 0;
  L.epoch++;
  L.work = 0;
  L.stall = 0;
  L.flow_ref = L.flow;
  L.fsel = L_FRONT;
  const unsigned f = L.fcnt + L.fcnth;
  if (f == 0 || L.after_gr_exit) L.state = ST_DONE;
  else L.state = f <= P.tail_enter ? ST_TAIL : round_state(P);
}

__device__ void advance(Sched& L, const Snap& q, const Params& P, const NetDev& N, Ctl* c) {
  switch (L.state) {
    case ST_ROUND_A:
      L.ncnt = q.c[C_NEXT];
      L.ncnth = q.c[C_NEXTH];
      L.flow += q.flow;
      L.state = ST_ROUND_B;
      break;
    case ST_ROUND_B: {
      const unsigned fprev = L.fcnt + L.fcnth, nprev = L.ncnt + L.ncnth;
      L.rounds++;
      L.work += (unsigned long long)fprev + nprev;
      L.fcnt = q.c[C_FRONT];
      L.fcnth = q.c[C_FRONTH];
      L.rcnt = q.c[C_RELAB];
      L.lp ^= 1;
      L.epoch++;
      const unsigned f = L.fcnt + L.fcnth;
      if (L.flow != L.flow_ref || f >= P.stall_nodes) {
        L.flow_ref = L.flow;
        L.stall = 0;
      } else {
        L.stall++;
      }
      if (f == 0) {
        begin_gr(L);
      } else if (L.rounds >= P.max_rounds) {
        atomicCAS(&c->err, kDevOk, kDevIterLimit);
        L.state = ST_DONE;
      } else if (L.work >= P.gr_work || L.stall >= stall_limit(L, P)) {
        begin_gr(L);
      } else {
        L.state = f <= P.tail_enter ? ST_TAIL : ST_ROUND_A;
      }
      break;
    }
    case ST_ROUND: {
      // one-phase round: the next frontier is the list this round filled
      const unsigned fprev = L.fcnt + L.fcnth;
      L.flow += q.flow;
      L.rounds++;
      L.fcnt = q.c[C_NEXT];
      L.fcnth = q.c[C_NEXTH];
      L.work += (unsigned long long)fprev + L.fcnt + L.fcnth;
      L.fsel ^= 1;
      L.lp ^= 1;
      L.epoch++;
      const unsigned f = L.fcnt + L.fcnth;
      if (L.flow != L.flow_ref || f >= P.stall_nodes) {
        L.flow_ref = L.flow;
        L.stall = 0;
      } else {
        L.stall++;
      }
      if (f == 0) {
        begin_gr(L);   // nothing was pushed: no pending deltas
      } else if (L.rounds >= P.max_rounds) {
        atomicCAS(&c->err, kDevOk, kDevIterLimit);
        L.state = ST_DONE;
      } else if (L.work >= P.gr_work || L.stall >= stall_limit(L, P)) {
        L.state = ST_FLUSH;
      } else {
        L.state = f <= P.tail_enter ? ST_TAIL : ST_ROUND;
      }
      break;
    }
    case ST_FLUSH:
      begin_gr(L);
      break;
    case ST_GR_SEED:
      L.state = ST_GR_RUN;
      break;
    case ST_GR_RUN:
      L.gq_items += q.gq_tail;
      L.gq_prev = q.gq_tail;
      if (q.gq_over) {
        L.gq_overs++;
        // the queue overflowed: redo this global relabel level by level
        L.gr_sync = 1;
        L.wT = 0;
        L.state = ST_GR_INIT;
      } else {
        L.gr_levels += (unsigned long long)q.gq_maxd + 1;
        L.wT += q.w;
        end_gr(L, q, P, q.gq_maxd + 1);
      }
      break;
    case ST_GR_INIT:
    case ST_GR_ADD:
    case ST_SR_INIT:
    case ST_SR_ADD:
    case ST_DIST_INIT:
      L.bfs_begin = 0;
      L.bfs_end = q.c[C_BFS];
      L.bfsh_begin = 0;
      L.bfsh_end = q.c[C_BFSH];
      L.level = 0;
      if (L.state == ST_GR_INIT || L.state == ST_GR_ADD) L.wT += q.w;
      if (L.state == ST_SR_INIT || L.state == ST_SR_ADD) L.wS += q.w;
      if (L.state == ST_GR_INIT && P.async_gr && N.gq && !L.gr_sync) {
        L.state = ST_GR_SEED;   // the sinks (this phase's BFS list) seed the queue
        break;
      }
      L.state = (L.state == ST_GR_INIT || L.state == ST_GR_ADD) ? ST_GR_LEVEL
                : L.state == ST_DIST_INIT ? ST_DIST_LEVEL : ST_SR_LEVEL;
      break;
    case ST_GR_LEVEL:
    case ST_SR_LEVEL:
    case ST_DIST_LEVEL: {
      const int st = L.state;
      if (st == ST_GR_LEVEL) {
        L.gr_levels++;
        L.wT += q.w;
      }
      if (st == ST_SR_LEVEL) L.wS += q.w;
      if (q.c[C_BFS] == 0 && q.c[C_BFSH] == 0) {
        if (st == ST_GR_LEVEL) {
          end_gr(L, q, P, (unsigned)L.level + 1);
        } else {
          L.epoch++;
          L.state = ST_DONE;
        }
      } else {
        L.bfs_begin = L.bfs_end;
        L.bfs_end += q.c[C_BFS];
        L.bfsh_begin = L.bfsh_end;
        L.bfsh_end += q.c[C_BFSH];
        L.level++;
      }
      break;
    }
    default:
      L.state = ST_DONE;
  }
}

__device__ __forceinline__ unsigned ld_cg(const unsigned* p) { return *(const volatile unsigned*)p; }

// Snapshot of the counters of the phase with index k (slot k % 3).
__device__ Snap take_snap(EngineCtl* E, unsigned k) {
  const unsigned sl = k % 3;
  Snap q;
#pragma unroll
  for (int i = 0; i < C_COUNT; i++) q.c[i] = ld_cg(&E->cnt3[i][sl]);
  q.act = ld_cg(&E->gr_act[0]);
  q.acth = ld_cg(&E->gr_act[1]);
  q.flow = *(const volatile unsigned long long*)&E->flow3[sl];
  q.w = *(const volatile long long*)&E->w3[sl];
  q.key = *(const volatile unsigned long long*)&E->key3[sl];
  q.node = *(const volatile int*)&E->node3[sl];
  q.gq_over = ld_cg(&E->gq_over);
  q.gq_maxd = ld_cg(&E->gq_maxd);
  q.gq_tail = ld_cg(&E->gq_tail);
  return q;
}

// Zero the slot the next phase will append to.  Only CTA 0 does it (stores
// of every CTA to the same lines cost more than the whole barrier); the slot
// was last read before the previous barrier and is next appended to after
// the coming one.
__device__ __forceinline__ void clear_slot(EngineCtl* E, unsigned sl, bool gr_init) {
  for (int l = 0; l < C_COUNT; l++) E->cnt3[l][sl] = 0;
  E->flow3[sl] = 0;
  E->w3[sl] = 0;
  E->key3[sl] = 0;
  E->node3[sl] = -1;
  if (gr_init) {
    E->gr_act[0] = 0;
    E->gr_act[1] = 0;
  }
}

// Count-up grid barrier for a cooperative launch (all CTAs co-resident): a
// CTA adds one and waits until every CTA has added one for this barrier.  The
// arrival is a release reduction and the wait an acquire spin, so the writes
// of every CTA before the barrier are visible to every CTA after it.  The
// wait is bounded by timeout_ns of globaltimer: on expiry, or when it finds
// ctl->err raised by another CTA (polled every 256 spins), ctl->err is set and
// false is returned.  A CTA that raised an error itself also moves its own
// schedule to ST_DONE, so no error needs to be read after a completed wait.
__device__ bool grid_barrier(EngineCtl* E, unsigned target, unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(&E->bar_count, 1u);
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (!count_reached(ld_acquire(&E->bar_count), target)) {
      if ((++spins & 255u) == 0) {
        if (ld_volatile_int(&E->c.err) != kDevOk) { ok = 0; break; }
        const unsigned long long t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > timeout_ns) {
          atomicCAS(&E->c.err, kDevOk, kDevTimeout);
          E->c.err_where = 1;
          ok = 0;
          break;
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------------------
// push delivery: returns true when y must join the next list
__device__ __forceinline__ bool deliver(const NetDev& N, int y, long long d, unsigned epoch,
                                        long long& sink_acc, bool& heavy) {
  const uint8_t fl = N.flags[y];
  heavy = (fl & kHeavy) != 0;
  if (fl & kSink) {
    sink_acc += d;
    return false;
  }
  if (fl & kSource) return false;
  atomicAdd((unsigned long long*)&N.delta[y], (unsigned long long)d);
  return atomicExch(&N.stamp[y], epoch) != epoch;
}

// Team primitives: a team is TW consecutive lanes of a warp (TW = 8 for light
// nodes, 32 for heavy ones); every lane of the warp must take part.
template <int TW>
__device__ __forceinline__ long long team_incl_scan(long long v, unsigned tl) {
#pragma unroll
  for (int o = 1; o < TW; o <<= 1) {
    const long long t = __shfl_up_sync(FULL, v, o, TW);
    if ((int)tl >= o) v += t;
  }
  return v;
}

template <int TW>
__device__ __forceinline__ int team_min(int v) {
#pragma unroll
  for (int o = TW / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o, TW));
  return v;
}

// Discharge of one node by a team of TW lanes (Section 8.1: one scan of the
// node's residual arcs in arc order; push min(excess, residual) on every
// admissible arc until the excess is gone).  TW arc groups per step; pushes
// are placed by an inclusive scan of residual capacities.  x < 0: idle team.
template <int TW>
__device__ void discharge_team(const NetDev& N, int x, const int32_t* Lr, unsigned epoch,
                               unsigned lane, long long& sink_acc, Acc& a, const Slot& S) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  const unsigned tl = lane & (TW - 1);
  long long rem = 0;
  int dx = NL;
  if (x >= 0) {
    rem = __ldcg(&N.excess[x]);   // may come from atomics (saturation)
    dx = Lr[x];
  }
  const bool act = x >= 0 && rem > 0 && dx < NL;
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  if (act) {
    g = node_arcs(N, x);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
  } else {
    rem = 0;
  }
  const int dt = dx - 1;
  const unsigned steps = warp_max_u((g.items + TW - 1) / TW);
  int32_t* nl = N.list[L_NEXT];
  for (unsigned c = 0; c < steps; c++) {
    const unsigned k = c * TW + tl;
    long long r1 = 0, r2 = 0;
    int y1 = -1, y2 = -1, p = 0, fi = 0, fo = 0;
    if (rem > 0 && k < g.items) {
      if (g.kind == 0) {
        // hypernode: (u, e_in) with residual w(e) - f_in, (u, e_out) with f_out
        const int2 it = N.inc[g.beg + k];
        p = it.y;
        const int ww = N.net_w[it.x];
        fi = N.f_in[p];
        fo = N.f_out[p];
        y1 = nh + it.x;
        y2 = nh + m + it.x;
        if (ww > fi && Lr[y1] == dt) r1 = ww - fi;
        if (fo > 0 && Lr[y2] == dt) r2 = fo;
        a.hyper++;
      } else if (g.kind == 1) {
        // in-node: bridge (e_in, e_out) with residual w - f_b; (e_in, u) with f_in
        if (k == 0) {
          y1 = nh + m + g.e;
          if (w > fb && Lr[y1] == dt) r1 = w - fb;
        } else {
          p = g.beg + k - 1;
          fi = N.f_in[p];
          if (fi > 0) {
            y1 = N.pin[p];
            if (Lr[y1] == dt) r1 = fi;
          }
        }
        a.net++;
      } else {
        // out-node: (e_out, e_in) with residual f_b; (e_out, u) uncapacitated
        if (k == 0) {
          y1 = nh + g.e;
          if (fb > 0 && Lr[y1] == dt) r1 = fb;
        } else {
          p = g.beg + k - 1;
          y1 = N.pin[p];
          if (Lr[y1] == dt) r1 = rem;
        }
        a.net++;
      }
    }
    const long long r = r1 + r2;
    const long long incl = team_incl_scan<TW>(r, tl);
    const long long take = min(max(rem - (incl - r), 0LL), r);
    const long long t1 = min(take, r1), t2 = take - t1;
    bool a1 = false, a2 = false, h1 = false, h2 = false;
    if (t1 > 0) {
      if (g.kind == 0) N.f_in[p] = fi + (int)t1;
      else if (g.kind == 1) {
        if (k == 0) N.f_b[g.e] = fb + (int)t1;
        else N.f_in[p] = fi - (int)t1;
      } else {
        if (k == 0) N.f_b[g.e] = fb - (int)t1;
        else N.f_out[p] += (int)t1;
      }
      a1 = deliver(N, y1, t1, epoch, sink_acc, h1);
      a.pushes++;
    }
    if (t2 > 0) {
      N.f_out[p] = fo - (int)t2;
      a2 = deliver(N, y2, t2, epoch, sink_acc, h2);
      a.pushes++;
    }
    append_split(a1, y1, h1, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    append_split(a2, y2, h2, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    const long long tot = __shfl_sync(FULL, incl, TW - 1, TW);
    rem -= min(rem, tot);
  }
  bool want = false;
  if (act && tl == 0) {
    N.excess[x] = rem;
    if (rem > 0) {
      N.needrl[x] = 1;
      want = atomicExch(&N.stamp[x], epoch) != epoch;
    }
    a.nodes++;
  }
  append_split(want, x, TW == 32, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
}

// New label after the pushes of the round: min over residual arcs (capped
// network) of d(v) + 1 with the labels of the round (Section 2, "relabel");
// NL when no residual arc is left.  One node per team (need = false: idle).
template <int TW>
__device__ int relabel_team(const NetDev& N, const int32_t* Lr, int x, bool need, unsigned lane,
                            Acc& a) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  const unsigned tl = lane & (TW - 1);
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  if (need) {
    g = node_arcs(N, x);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
  }
  const unsigned steps = warp_max_u((g.items + TW - 1) / TW);
  int best = NL;
  for (unsigned c = 0; c < steps; c++) {
    const unsigned k = c * TW + tl;
    if (k >= g.items) continue;
    if (g.kind == 0) {
      const int2 it = N.inc[g.beg + k];
      if (N.net_w[it.x] > N.f_in[it.y]) best = min(best, Lr[nh + it.x] + 1);
      if (N.f_out[it.y] > 0) best = min(best, Lr[nh + m + it.x] + 1);
      a.hyper++;
    } else if (k == 0) {
      if (g.kind == 1 ? w > fb : fb > 0)
        best = min(best, Lr[g.kind == 1 ? nh + m + g.e : nh + g.e] + 1);
      a.net++;
    } else {
      const unsigned p = g.beg + k - 1;
      if (g.kind == 2 || N.f_in[p] > 0) best = min(best, Lr[N.pin[p]] + 1);
      a.net++;
    }
  }
  best = team_min<TW>(best);
  return min(best, NL);
}

// ---------------------------------------------------------------------------
// Heavy nodes: a whole CTA per node.  Block-wide inclusive scan of one value
// per thread; *total gets the sum.  Every thread of the CTA must call it.
__device__ __forceinline__ long long block_incl_scan(long long v, long long* total) {
  __shared__ long long wtot[32];
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  long long x = warp_incl_scan(v);
  if (lane == 31) wtot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const long long t = lane < nw ? wtot[lane] : 0;
    const long long y = warp_incl_scan(t);
    if (lane < nw) wtot[lane] = y - t;
    if (lane == nw - 1) wtot[31] = y;
  }
  __syncthreads();
  x += wtot[wid];
  *total = wtot[31];
  __syncthreads();
  return x;
}

__device__ __forceinline__ int block_min(int v) {
  __shared__ int wmin[32];
  const unsigned lane = lane_id(), wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_min(v);
  if (lane == 0) wmin[wid] = v;
  __syncthreads();
  if (wid == 0) {
    int t = lane < nw ? wmin[lane] : INT_MAX;
    t = warp_min(t);
    if (lane == 0) wmin[31] = t;
  }
  __syncthreads();
  const int r = wmin[31];
  __syncthreads();
  return r;
}

// Discharge of one heavy node by the whole CTA: blockDim.x arc groups per
// step, pushes placed by a block scan of residual capacities in arc order.
__device__ void discharge_block(const NetDev& N, int x, const int32_t* Lr, unsigned epoch,
                                long long& sink_acc, Acc& a, const Slot& S) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  const long long ex = __ldcg(&N.excess[x]);   // may come from atomics (saturation)
  const int dx = Lr[x];
  if (ex <= 0 || dx >= NL) return;    // uniform over the CTA
  const int dt = dx - 1;
  long long rem = ex;
  int32_t* nl = N.list[L_NEXT];
  const NodeArcs g = node_arcs(N, x);
  const int w = g.kind ? N.net_w[g.e] : 0;
  const int fb = g.kind ? N.f_b[g.e] : 0;
  for (unsigned k0 = 0; k0 < g.items && rem > 0; k0 += blockDim.x) {
    const unsigned k = k0 + threadIdx.x;
    long long r1 = 0, r2 = 0;
    int y1 = -1, y2 = -1, p = 0, fi = 0, fo = 0;
    if (k < g.items) {
      if (g.kind == 0) {
        const int2 it = N.inc[g.beg + k];
        p = it.y;
        const int ww = N.net_w[it.x];
        fi = N.f_in[p];
        fo = N.f_out[p];
        y1 = nh + it.x;
        y2 = nh + m + it.x;
        if (ww > fi && Lr[y1] == dt) r1 = ww - fi;
        if (fo > 0 && Lr[y2] == dt) r2 = fo;
        a.hyper++;
      } else if (g.kind == 1) {
        if (k == 0) {
          y1 = nh + m + g.e;
          if (w > fb && Lr[y1] == dt) r1 = w - fb;
        } else {
          p = g.beg + k - 1;
          fi = N.f_in[p];
          if (fi > 0) {
            y1 = N.pin[p];
            if (Lr[y1] == dt) r1 = fi;
          }
        }
        a.net++;
      } else {
        if (k == 0) {
          y1 = nh + g.e;
          if (fb > 0 && Lr[y1] == dt) r1 = fb;
        } else {
          p = g.beg + k - 1;
          y1 = N.pin[p];
          if (Lr[y1] == dt) r1 = rem;
        }
        a.net++;
      }
    }
    const long long r = r1 + r2;
    long long tot;
    const long long incl = block_incl_scan(r, &tot);
    const long long take = min(max(rem - (incl - r), 0LL), r);
    const long long t1 = min(take, r1), t2 = take - t1;
    bool a1 = false, a2 = false, h1 = false, h2 = false;
    if (t1 > 0) {
      if (g.kind == 0) N.f_in[p] = fi + (int)t1;
      else if (g.kind == 1) {
        if (k == 0) N.f_b[g.e] = fb + (int)t1;
        else N.f_in[p] = fi - (int)t1;
      } else {
        if (k == 0) N.f_b[g.e] = fb - (int)t1;
        else N.f_out[p] += (int)t1;
      }
      a1 = deliver(N, y1, t1, epoch, sink_acc, h1);
      a.pushes++;
    }
    if (t2 > 0) {
      N.f_out[p] = fo - (int)t2;
      a2 = deliver(N, y2, t2, epoch, sink_acc, h2);
      a.pushes++;
    }
    append_split(a1, y1, h1, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    append_split(a2, y2, h2, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    rem -= min(rem, tot);
  }
  bool want = false;
  if (threadIdx.x == 0) {
    N.excess[x] = rem;
    if (rem > 0) {
      N.needrl[x] = 1;
      want = atomicExch(&N.stamp[x], epoch) != epoch;
    }
    a.nodes++;
  }
  if (threadIdx.x < 32) append_split(want, x, true, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
}

// Relabel of one heavy node by the whole CTA (see relabel_team).
__device__ int relabel_block(const NetDev& N, const int32_t* Lr, int x, Acc& a) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  const NodeArcs g = node_arcs(N, x);
  int best = NL;
  for (unsigned k = threadIdx.x; k < g.items; k += blockDim.x) {
    if (g.kind == 0) {
      const int2 it = N.inc[g.beg + k];
      if (N.net_w[it.x] > N.f_in[it.y]) best = min(best, Lr[nh + it.x] + 1);
      if (N.f_out[it.y] > 0) best = min(best, Lr[nh + m + it.x] + 1);
      a.hyper++;
    } else if (k == 0) {
      const int w = N.net_w[g.e], fb = N.f_b[g.e];
      if (g.kind == 1 ? w > fb : fb > 0)
        best = min(best, Lr[g.kind == 1 ? nh + m + g.e : nh + g.e] + 1);
      a.net++;
    } else {
      const unsigned p = g.beg + k - 1;
      if (g.kind == 2 || N.f_in[p] > 0) best = min(best, Lr[N.pin[p]] + 1);
      a.net++;
    }
  }
  return min(block_min(best), NL);
}

// delta[] only grows by atomics, which update L2, not the L1 copy a previous
// round's load of the same line may have left on this SM; between the phases
// of a CTA-alone round (block barriers, no GPU-scope fence) a cached load
// could return the old value and drop pushed excess.  Hence the L2 load.
__device__ __forceinline__ long long apply_delta(const NetDev& N, int y) {
  const long long d = __ldcg(&N.delta[y]);
  const long long ex = N.excess[y] + d;
  if (d) N.delta[y] = 0;
  N.excess[y] = ex;
  return ex;
}

// Phase B for one heavy node by the whole CTA.
__device__ void apply_relabel_block(const NetDev& N, const int32_t* Lr, int32_t* Ln, int y,
                                    Acc& a, const Slot& S) {
  __shared__ int s_need;
  __shared__ long long s_ex;
  const int NL = N.NL;
  if (threadIdx.x == 0) {
    s_ex = apply_delta(N, y);
    s_need = N.needrl[y];
    if (s_need) N.needrl[y] = 0;
    a.nodes++;
  }
  __syncthreads();
  const int need = s_need;
  const long long ex = s_ex;
  int lab = 0;
  if (need) {
    lab = relabel_block(N, Lr, y, a);
    if (threadIdx.x == 0) Ln[y] = lab;
  } else {
    lab = Lr[y];
  }
  if (threadIdx.x < 32) {
    append_plain(threadIdx.x == 0 && need, y, N.list[L_RELAB], S.c[C_RELAB], 0);
    append_split(threadIdx.x == 0 && ex > 0 && lab < NL, y, true, N.list[L_FRONT], S.c[C_FRONT],
                 S.c[C_FRONTH], 0, 0, NL);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
__device__ void phase_a(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                        unsigned lane, Acc& a, EngineCtl* E) {
  const int32_t* Lr = lab_cur(N, L.lp);
  int32_t* Ln = lab_cur(N, L.lp ^ 1);
  for (unsigned i = T.tid; i < L.rcnt; i += T.nth) {   // labels relabeled last round
    const int x = N.list[L_RELAB][i];
    Ln[x] = Lr[x];
  }
  long long sink_acc = 0;
  const int32_t* fl = N.list[L_FRONT];
  constexpr unsigned TPW = 32 / kTeam;                 // light nodes per warp
  for (unsigned base = T.gwarp * TPW; base < L.fcnt; base += T.nwarps * TPW) {
    const unsigned i = base + lane / kTeam;
    discharge_team<kTeam>(N, i < L.fcnt ? fl[i] : -1, Lr, L.epoch, lane, sink_acc, a, S);
  }
  for (unsigned h = T.block; h < L.fcnth; h += T.nblocks)
    discharge_block(N, fl[N.NL - 1 - h], Lr, L.epoch, sink_acc, a, S);
  sink_acc = warp_sum(sink_acc);
  if (lane == 0 && sink_acc) atomicAdd(S.flow, (unsigned long long)sink_acc);
}

// Phase B for the entry of one team: apply the round's excess delta and, if
// the node kept excess after its pushes, relabel it.
template <int TW>
__device__ void apply_relabel_team(const NetDev& N, const int32_t* Lr, int32_t* Ln, int y,
                                   unsigned lane, Acc& a, const Slot& S) {
  const int NL = N.NL;
  const unsigned tl = lane & (TW - 1);
  long long ex = 0;
  int need = 0, lab = NL;
  if (y >= 0 && tl == 0) {
    ex = apply_delta(N, y);
    lab = Lr[y];
    need = N.needrl[y];
    if (need) N.needrl[y] = 0;
    a.nodes++;
  }
  need = __shfl_sync(FULL, need, 0, TW);
  const int nl = relabel_team<TW>(N, Lr, y, need != 0, lane, a);
  if (need && tl == 0) {
    lab = nl;
    Ln[y] = nl;
  }
  append_plain(tl == 0 && need, y, N.list[L_RELAB], S.c[C_RELAB], 0);
  append_split(tl == 0 && y >= 0 && ex > 0 && lab < NL, y, TW == 32, N.list[L_FRONT],
               S.c[C_FRONT], S.c[C_FRONTH], 0, 0, NL);
}

__device__ void phase_b(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                        unsigned lane, Acc& a) {
  const int32_t* Lr = lab_cur(N, L.lp);
  int32_t* Ln = lab_cur(N, L.lp ^ 1);
  const int32_t* nx = N.list[L_NEXT];
  constexpr unsigned TPW = 32 / kTeam;
  for (unsigned base = T.gwarp * TPW; base < L.ncnt; base += T.nwarps * TPW) {
    const unsigned i = base + lane / kTeam;
    apply_relabel_team<kTeam>(N, Lr, Ln, i < L.ncnt ? nx[i] : -1, lane, a, S);
  }
  for (unsigned h = T.block; h < L.ncnth; h += T.nblocks)
    apply_relabel_block(N, Lr, Ln, nx[N.NL - 1 - h], a, S);
}

// ---------------------------------------------------------------------------
// One-phase rounds.  The two-phase round above spends a grid barrier and a
// second dependent load chain on applying deltas and relabelling.  Here a
// round is one phase: every frontier node first applies the pushes it
// received in the previous round (delta buffers alternate by round parity,
// so this round's pushes never mix with them), discharges against the labels
// of the round, and relabels itself at once from its own arcs:
//   new label = min(min over its residual arcs (x, y) of d(y) + 1, d(x) + 2).
// The first term is the usual relabel over the arcs left residual by x's own
// pushes (read with the round's labels, which only grow, so it stays valid
// when neighbours relabel too).  The arcs that other nodes' pushes open into
// x this round come from nodes with label d(x) + 1, so they never ask for
// more than d(x) + 2; capping at d(x) + 2 keeps the labelling valid without
// knowing whether such pushes happened.  It never exceeds the two-phase
// relabel and still raises the label by at least one (no admissible arc is
// left), so the method and its results are those of push-relabel; only the
// number of rounds can differ.  Labels stay double-buffered: a node writes
// its next label only when it is in the frontier, and every node whose label
// changes keeps excess, so it is in the next frontier and copies its label
// into the other buffer there.

// A round's delta word of a node doubles as its membership of the next
// frontier: the first addition (a push, or kSelf by a node that keeps
// excess) finds zero and appends the node.  Readers strip kSelf.
constexpr long long kSelf = 1ll << 62;

__device__ __forceinline__ long long strip_self(long long d) { return d & ~kSelf; }

// Push of d into y (flag byte fl of y, loaded with its label).  Returns true
// when y must join the next frontier.
__device__ __forceinline__ bool deliver_to(long long* dcur, int y, uint8_t fl, long long d,
                                           long long& sink_acc) {
  if (fl & kSink) {
    sink_acc += d;
    return false;
  }
  if (fl & kSource) return false;
  return atomicAdd((unsigned long long*)&dcur[y], (unsigned long long)d) == 0ull;
}

// Arc group k of node x for a discharge with relabel: admissible residuals
// r1, r2 (label dt), residual capacities q1, q2 (-1: none; kInfRes: the
// uncapacitated (e_out, u)) and head labels l1, l2.
constexpr long long kInfRes = 1ll << 62;

__device__ __forceinline__ void arc_group(const NetDev& N, const NodeArcs& g, unsigned k, int w,
                                          int fb, const int32_t* Lr, int dt, long long rem,
                                          long long& r1, long long& r2, long long& q1,
                                          long long& q2, int& l1, int& l2, int& y1, int& y2,
                                          uint8_t& f1, uint8_t& f2, int& p, int& fi, int& fo,
                                          Acc& a) {
  const int nh = N.n_nodes, m = N.m_nets;
  if (g.kind == 0) {
    const int2 it = N.inc[g.beg + k];
    p = it.y;
    const int ww = N.net_w[it.x];
    fi = N.f_in[p];
    fo = N.f_out[p];
    y1 = nh + it.x;
    y2 = nh + m + it.x;
    l1 = Lr[y1];
    l2 = Lr[y2];
    f1 = N.flags[y1];
    f2 = N.flags[y2];
    q1 = ww - fi;
    q2 = fo;
    if (q1 > 0 && l1 == dt) r1 = q1;
    if (q2 > 0 && l2 == dt) r2 = q2;
    a.hyper++;
  } else if (g.kind == 1) {
    if (k == 0) {
      y1 = nh + m + g.e;
      q1 = w - fb;
      l1 = Lr[y1];
      f1 = N.flags[y1];
      if (q1 > 0 && l1 == dt) r1 = q1;
    } else {
      p = g.beg + k - 1;
      fi = N.f_in[p];
      const int u = N.pin[p];
      q1 = fi;
      if (fi > 0) {
        y1 = u;
        l1 = Lr[y1];
        f1 = N.flags[y1];
        if (l1 == dt) r1 = fi;
      }
    }
    a.net++;
  } else {
    if (k == 0) {
      y1 = nh + g.e;
      q1 = fb;
      if (fb > 0) {
        l1 = Lr[y1];
        f1 = N.flags[y1];
        if (l1 == dt) r1 = fb;
      }
    } else {
      p = g.beg + k - 1;
      y1 = N.pin[p];
      l1 = Lr[y1];
      f1 = N.flags[y1];
      q1 = kInfRes;
      if (l1 == dt) r1 = rem;
    }
    a.net++;
  }
}

// Flow updates of the takes t1, t2 on arc group k (as in discharge_team).
__device__ __forceinline__ void apply_takes(const NetDev& N, const NodeArcs& g, unsigned k,
                                            int fb, int p, int fi, int fo, long long t1,
                                            long long t2) {
  if (t1 > 0) {
    if (g.kind == 0) N.f_in[p] = fi + (int)t1;
    else if (g.kind == 1) {
      if (k == 0) N.f_b[g.e] = fb + (int)t1;
      else N.f_in[p] = fi - (int)t1;
    } else {
      if (k == 0) N.f_b[g.e] = fb - (int)t1;
      else N.f_out[p] += (int)t1;
    }
  }
  if (t2 > 0) N.f_out[p] = fo - (int)t2;
}

// Relabel candidate of the arcs of one group after its takes.
__device__ __forceinline__ int group_cand(long long q1, long long q2, int l1, int l2,
                                          long long t1, long long t2, int cand) {
  if (q1 > 0 && q1 - t1 > 0) cand = min(cand, l1 + 1);
  if (q2 > 0 && q2 - t2 > 0) cand = min(cand, l2 + 1);
  return cand;
}

// ParPR-Block (Section 8.2, the first of the two fixes of the push-relabel
// conflict), the alternative to the capped self relabel of one-phase rounds:
// in round R a node that was pushed to may not relabel, and a node that
// relabeled may not be pushed to, whichever comes first.  Each node has a
// tag word; R's tags are 2R (pushed to) and 2R + 1 (relabeled), set by
// compare-and-swap, so the first of the two operations wins and the other is
// refused.  A refused push leaves the arc residual (the node keeps its
// excess for the next round); a refused relabel keeps the label.  The node
// then relabels to the plain minimum over its residual arcs, without the
// d(x) + 2 cap.  pb_mark(blk, y, mine, other) sets y's tag to `mine` unless
// it already holds `other`; true when y holds `mine` afterwards.
__device__ __forceinline__ bool pb_mark(uint32_t* blk, int y, unsigned mine, unsigned other) {
  unsigned cur = *(volatile uint32_t*)&blk[y];
  for (int i = 0; i < 3; i++) {
    if (cur == mine) return true;
    if (cur == other) return false;
    const unsigned old = atomicCAS(&blk[y], cur, mine);
    if (old == cur) return true;
    cur = old;   // another thread set one of this round's tags
  }
  return cur == mine;
}

// New label of a discharged node with excess left: the capped self relabel,
// or under ParPR-Block (pbt = 2R != 0) the uncapped one when x may relabel.
__device__ __forceinline__ int round_label(const NetDev& N, int x, int dx, int cand,
                                           unsigned pbt) {
  if (!pbt) return min(min(cand, dx + 2), N.NL);
  const int nl = min(cand, N.NL);
  if (nl > dx && !pb_mark(N.blk, x, pbt | 1u, pbt)) return dx;
  return nl;
}

// One-phase discharge of node x by a team of TW lanes (x < 0: idle team).
template <int TW>
__device__ void round_team(const NetDev& N, int x, const int32_t* Lr, int32_t* Ln,
                           long long* dprev, long long* dcur, int32_t* nl, unsigned lane,
                           long long& sink_acc, Acc& a, const Slot& S, unsigned pbt) {
  const int NL = N.NL;
  const unsigned tl = lane & (TW - 1);
  long long ex = 0, dp0 = 0;
  int dx = NL;
  if (x >= 0) {
    ex = __ldcg(&N.excess[x]);
    dp0 = __ldcg(&dprev[x]);
    dx = Lr[x];
  }
  const long long dp = strip_self(dp0);
  ex += dp;
  const bool act = x >= 0 && ex > 0 && dx < NL;
  long long rem = act ? ex : 0;
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  if (act) {
    g = node_arcs(N, x);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
  }
  const int dt = dx - 1;
  int cand = NL;
  const unsigned steps = warp_max_u((g.items + TW - 1) / TW);
  for (unsigned c = 0; c < steps; c++) {
    const unsigned k = c * TW + tl;
    long long r1 = 0, r2 = 0, q1 = -1, q2 = -1;
    int l1 = NL, l2 = NL, y1 = -1, y2 = -1, p = 0, fi = 0, fo = 0;
    uint8_t f1 = 0, f2 = 0;
    if (rem > 0 && k < g.items)
      arc_group(N, g, k, w, fb, Lr, dt, rem, r1, r2, q1, q2, l1, l2, y1, y2, f1, f2, p, fi, fo,
                a);
    if (pbt) {
      if (r1 > 0 && !(f1 & kTerminal) && !pb_mark(N.blk, y1, pbt, pbt | 1u)) r1 = 0;
      if (r2 > 0 && !(f2 & kTerminal) && !pb_mark(N.blk, y2, pbt, pbt | 1u)) r2 = 0;
    }
    const long long r = r1 + r2;
    const long long incl = team_incl_scan<TW>(r, tl);
    const long long take = min(max(rem - (incl - r), 0LL), r);
    const long long t1 = min(take, r1), t2 = take - t1;
    cand = group_cand(q1, q2, l1, l2, t1, t2, cand);
    apply_takes(N, g, k, fb, p, fi, fo, t1, t2);
    bool a1 = false, a2 = false;
    if (t1 > 0) {
      a1 = deliver_to(dcur, y1, f1, t1, sink_acc);
      a.pushes++;
    }
    if (t2 > 0) {
      a2 = deliver_to(dcur, y2, f2, t2, sink_acc);
      a.pushes++;
    }
    append_split(a1, y1, (f1 & kHeavy) != 0, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    append_split(a2, y2, (f2 & kHeavy) != 0, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    const long long tot = __shfl_sync(FULL, incl, TW - 1, TW);
    rem -= min(rem, tot);
  }
  cand = team_min<TW>(cand);
  bool want = false;
  if (x >= 0 && tl == 0) {
    if (dp || dp0) dprev[x] = 0;
    if (act) {
      N.excess[x] = rem;
      Ln[x] = rem > 0 ? round_label(N, x, dx, cand, pbt) : dx;
      if (rem > 0)
        want = atomicAdd((unsigned long long*)&dcur[x], (unsigned long long)kSelf) == 0ull;
      a.nodes++;
    } else {
      // no excess, or cut off from the sinks: keep the excess and the label
      if (dp) N.excess[x] = ex;
      Ln[x] = dx;
    }
  }
  append_split(want, x, TW == 32, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
}

// One-phase discharge of one heavy node by the whole CTA.
__device__ void round_block(const NetDev& N, int x, const int32_t* Lr, int32_t* Ln,
                            long long* dprev, long long* dcur, int32_t* nl, long long& sink_acc,
                            Acc& a, const Slot& S, unsigned pbt) {
  const int NL = N.NL;
  const long long dp0 = __ldcg(&dprev[x]);
  const long long dp = strip_self(dp0);
  const long long ex = __ldcg(&N.excess[x]) + dp;
  const int dx = Lr[x];
  if (ex <= 0 || dx >= NL) {   // uniform over the CTA
    __syncthreads();           // every thread has read dprev[x] before it is cleared
    if (threadIdx.x == 0) {
      if (dp0) dprev[x] = 0;
      if (dp) N.excess[x] = ex;
      Ln[x] = dx;
    }
    return;
  }
  const int dt = dx - 1;
  long long rem = ex;
  const NodeArcs g = node_arcs(N, x);
  const int w = g.kind ? N.net_w[g.e] : 0;
  const int fb = g.kind ? N.f_b[g.e] : 0;
  int cand = NL;
  for (unsigned k0 = 0; k0 < g.items && rem > 0; k0 += blockDim.x) {
    const unsigned k = k0 + threadIdx.x;
    long long r1 = 0, r2 = 0, q1 = -1, q2 = -1;
    int l1 = NL, l2 = NL, y1 = -1, y2 = -1, p = 0, fi = 0, fo = 0;
    uint8_t f1 = 0, f2 = 0;
    if (k < g.items)
      arc_group(N, g, k, w, fb, Lr, dt, rem, r1, r2, q1, q2, l1, l2, y1, y2, f1, f2, p, fi, fo,
                a);
    if (pbt) {
      if (r1 > 0 && !(f1 & kTerminal) && !pb_mark(N.blk, y1, pbt, pbt | 1u)) r1 = 0;
      if (r2 > 0 && !(f2 & kTerminal) && !pb_mark(N.blk, y2, pbt, pbt | 1u)) r2 = 0;
    }
    const long long r = r1 + r2;
    long long tot;
    const long long incl = block_incl_scan(r, &tot);
    const long long take = min(max(rem - (incl - r), 0LL), r);
    const long long t1 = min(take, r1), t2 = take - t1;
    cand = group_cand(q1, q2, l1, l2, t1, t2, cand);
    apply_takes(N, g, k, fb, p, fi, fo, t1, t2);
    bool a1 = false, a2 = false;
    if (t1 > 0) {
      a1 = deliver_to(dcur, y1, f1, t1, sink_acc);
      a.pushes++;
    }
    if (t2 > 0) {
      a2 = deliver_to(dcur, y2, f2, t2, sink_acc);
      a.pushes++;
    }
    append_split(a1, y1, (f1 & kHeavy) != 0, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    append_split(a2, y2, (f2 & kHeavy) != 0, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
    rem -= min(rem, tot);
  }
  cand = block_min(cand);
  bool want = false;
  if (threadIdx.x == 0) {
    if (dp0) dprev[x] = 0;
    N.excess[x] = rem;
    Ln[x] = rem > 0 ? round_label(N, x, dx, cand, pbt) : dx;
    if (rem > 0)
      want = atomicAdd((unsigned long long*)&dcur[x], (unsigned long long)kSelf) == 0ull;
    a.nodes++;
  }
  if (threadIdx.x < 32) append_split(want, x, true, nl, S.c[C_NEXT], S.c[C_NEXTH], 0, 0, NL);
}

// Delta buffers of round `rounds`: pushes go to cur, the previous round's
// pushes are read from prev.
__device__ __forceinline__ long long* delta_cur(const NetDev& N, unsigned long long rounds) {
  return (rounds & 1) ? N.delta1 : N.delta;
}
__device__ __forceinline__ long long* delta_prev(const NetDev& N, unsigned long long rounds) {
  return (rounds & 1) ? N.delta : N.delta1;
}

__device__ void phase_round(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                            unsigned lane, Acc& a, const Params& P) {
  // ParPR-Block tags of this round (0: capped self relabel)
  const unsigned pbt =
      P.parpr_block && N.blk ? (((unsigned)(L.rounds + 1) & 0x3fffffffu) << 1) : 0u;
  const int32_t* Lr = lab_cur(N, L.lp);
  int32_t* Ln = lab_cur(N, L.lp ^ 1);
  long long* dcur = delta_cur(N, L.rounds);
  long long* dprev = delta_prev(N, L.rounds);
  const int32_t* fl = N.list[L.fsel];
  int32_t* nl = N.list[L.fsel ^ 1];
  long long sink_acc = 0;
  constexpr unsigned TPW = 32 / kTeam;
  // While heavy nodes fill at most half of the CTAs, the last fcnth CTAs take
  // one heavy node each and no light ones, so that a heavy node's longer
  // chain runs beside the light work instead of after it.
  const unsigned nwb = blockDim.x >> 5;
  const bool split = L.fcnth > 0 && 2 * L.fcnth <= T.nblocks;
  const unsigned light_blocks = split ? T.nblocks - L.fcnth : T.nblocks;
  if (T.block < light_blocks) {
    const unsigned w0 = T.block * nwb + (threadIdx.x >> 5), nw = light_blocks * nwb;
    for (unsigned base = w0 * TPW; base < L.fcnt; base += nw * TPW) {
      const unsigned i = base + lane / kTeam;
      round_team<kTeam>(N, i < L.fcnt ? fl[i] : -1, Lr, Ln, dprev, dcur, nl, lane, sink_acc, a,
                        S, pbt);
    }
  }
  if (split) {
    if (T.block >= light_blocks)
      round_block(N, fl[N.NL - 1 - (T.block - light_blocks)], Lr, Ln, dprev, dcur, nl, sink_acc,
                  a, S, pbt);
  } else {
    for (unsigned h = T.block; h < L.fcnth; h += T.nblocks)
      round_block(N, fl[N.NL - 1 - h], Lr, Ln, dprev, dcur, nl, sink_acc, a, S, pbt);
  }
  sink_acc = warp_sum(sink_acc);
  if (lane == 0 && sink_acc) atomicAdd(S.flow, (unsigned long long)sink_acc);
}

// The last one-phase round's pushes are applied before a global relabel (the
// frontier list holds every node they reached).
__device__ void phase_flush(const NetDev& N, const Sched& L, const Team& T) {
  long long* dprev = delta_prev(N, L.rounds);
  const int32_t* fl = N.list[L.fsel];
  const unsigned tot = L.fcnt + L.fcnth;
  for (unsigned i = T.tid; i < tot; i += T.nth) {
    const int y = i < L.fcnt ? fl[i] : fl[N.NL - 1 - (i - L.fcnt)];
    const long long d = __ldcg(&dprev[y]);
    if (d) {
      N.excess[y] += strip_self(d);
      dprev[y] = 0;
    }
  }
}

// Global relabel, step 1: exact labels start from the sinks (Section 2,
// "global relabeling").
__device__ void gr_init(const NetDev& N, EngineCtl* E, const Sched& L, const Team& T,
                        const Slot& S, unsigned lane, Acc& a) {
  if (N.gq) {
    // empty the queue slots the last asynchronous relabel wrote
    const unsigned used = min(L.gq_prev, N.gq_cap);
    for (unsigned i = T.tid; i < used; i += T.nth) N.gq[i] = 0ull;
  }
  if (T.tid == 0) {
    // the work queue of an asynchronous relabel starts empty (nothing reads
    // it in this phase)
    E->gq_head = 0;
    E->gq_tail = 0;
    E->gq_done = 0;
    E->gq_over = 0;
    E->gq_maxd = 0;
  }
  for (unsigned x0 = T.tid - lane; x0 < (unsigned)N.NL; x0 += T.nth) {
    const unsigned x = x0 + lane;
    bool snk = false, hv = false;
    if (x < (unsigned)N.NL) {
      const uint8_t f = N.flags[x];
      snk = (f & kSink) != 0;
      hv = (f & kHeavy) != 0;
      const int l = snk ? 0 : N.NL;
      N.lab0[x] = l;
      N.lab1[x] = l;
      N.needrl[x] = 0;
      if (snk && x < (unsigned)N.n_nodes) a.w += N.node_w[x];
    }
    append_split(snk && (L.gr_one == 0 || (int)x == L.gr_one - 1), (int)x, hv, N.list[L_BFS],
                 S.c[C_BFS], S.c[C_BFSH], 0, 0, N.NL);
  }
}

// Sink-side cut after adding one sink u that no excess can reach (a piercing
// node outside S_r): the flow and S_r stay, T_r grows by the nodes that reach
// u, found by a reverse search seeded at u alone that only claims unlabelled
// nodes.  The labels of the old T_r are then no longer exact distances; the
// next flow computation starts with a full global relabel.
__device__ void gr_add(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                       unsigned lane, Acc& a) {
  if (T.tid >= 32) return;
  const int u = L.seed;
  bool seed = false, hv = false;
  if (lane == 0 && u >= 0) {
    N.lab0[u] = 0;
    N.lab1[u] = 0;
    hv = (N.flags[u] & kHeavy) != 0;
    if (u < N.n_nodes) a.w += N.node_w[u];
    seed = true;
  }
  append_split(seed, u, hv, N.list[L_BFS], S.c[C_BFS], S.c[C_BFSH], 0, 0, N.NL);
}

// Reverse residual arcs (capped network) into y, arc group k: up to two
// tails c1, c2 (-1 when none).
__device__ __forceinline__ void rev_arcs(const NetDev& N, const NodeArcs& g, unsigned k, int w,
                                         int fb, int& c1, int& c2, Acc& a) {
  const int nh = N.n_nodes, m = N.m_nets;
  c1 = c2 = -1;
  if (g.kind == 0) {
    // into a hypernode: (e_out, u) always, (e_in, u) when f_in > 0
    const int2 it = N.inc[g.beg + k];
    c1 = nh + m + it.x;
    if (N.f_in[it.y] > 0) c2 = nh + it.x;
    a.hyper++;
  } else if (k == 0) {
    // into e_in: (e_out, e_in) when f_b > 0; into e_out: bridge when w > f_b
    if (g.kind == 1) {
      if (fb > 0) c1 = nh + m + g.e;
    } else if (w > fb) {
      c1 = nh + g.e;
    }
  } else {
    // into e_in: (u, e_in) when f_in < w (capped); into e_out: (u, e_out) when f_out > 0
    const unsigned p = g.beg + k - 1;
    if (g.kind == 1 ? (N.f_in[p] < w) : (N.f_out[p] > 0)) c1 = N.pin[p];
    a.net++;
  }
}

// The tails c[0 .. K) of K arc groups (-1: none; a node may appear twice)
// claimed with label d1: a node still unlabelled (label N_L) that is not a
// source takes d1 by compare-and-swap (the one winning swap decides), joins
// the next level, T_r's weight, and the frontier when it has excess.  The
// loads of all K are issued before any claim, and the appends go in ballot
// passes of two per lane.
template <int K>
__device__ __forceinline__ void gr_emit(const NetDev& N, const Sched& L, const Slot& S,
                                        const int (&c)[K], int d1, Acc& a) {
  const int NL = N.NL;
  int l[K];
  uint8_t f[K];
  bool k[K], act[K], h[K];
#pragma unroll
  for (int i = 0; i < K; i++) {
    l[i] = 0;
    f[i] = 0;
    if (c[i] >= 0) {
      l[i] = N.lab0[c[i]];
      f[i] = N.flags[c[i]];
    }
  }
#pragma unroll
  for (int i = 0; i < K; i++) {
    k[i] = c[i] >= 0 && l[i] == NL && !(f[i] & kSource);
    if (k[i]) k[i] = atomicCAS(&N.lab0[c[i]], NL, d1) == NL;
  }
#pragma unroll
  for (int i = 0; i < K; i++) {
    act[i] = false;
    h[i] = (f[i] & kHeavy) != 0;
    if (k[i]) {
      N.lab1[c[i]] = d1;
      act[i] = N.excess[c[i]] > 0;
      if (c[i] < N.n_nodes) a.w += N.node_w[c[i]];
    }
  }
#pragma unroll
  for (int i = 0; i < K; i += 2) {
    append_split2(k[i], c[i], h[i], k[i + 1], c[i + 1], h[i + 1], N.list[L_BFS], S.c[C_BFS],
                  S.c[C_BFSH], L.bfs_end, L.bfsh_end, NL);
    append_split2(act[i], c[i], h[i], act[i + 1], c[i + 1], h[i + 1], N.list[L_FRONT], S.act[0],
                  S.act[1], 0, 0, NL);
  }
}

// Global relabel, one level: reverse BFS over residual arcs of the capped
// network; newly reached excess nodes become the frontier.  Light nodes by
// level_light, heavy ones by block_walk_heavy.
__device__ void gr_level(const NetDev& N, EngineCtl* E, const Sched& L, const Team& T,
                         const Slot& S, unsigned lane, Acc& a) {
  const int d1 = L.level + 1;
  const int32_t* bl = N.list[L_BFS];
  const unsigned nlight = L.bfs_end - L.bfs_begin, nheavy = L.bfsh_end - L.bfsh_begin;
  auto one = [&](const NodeArcs& g, unsigned k, int w, int fb) {
    int c[2] = {-1, -1};
    if (k != kNoArc) rev_arcs(N, g, k, w, fb, c[0], c[1], a);
    gr_emit<2>(N, L, S, c, d1, a);
  };
  auto two = [&](const WalkArc& A, const WalkArc& B) {
    int c[4] = {-1, -1, -1, -1};
    if (A.k != kNoArc) rev_arcs(N, A.g, A.k, A.w, A.fb, c[0], c[1], a);
    if (B.k != kNoArc) rev_arcs(N, B.g, B.k, B.w, B.fb, c[2], c[3], a);
    gr_emit<4>(N, L, S, c, d1, a);
  };
  level_light(N, bl + L.bfs_begin, nlight, T, lane, S.c[C_RELAB], one, two);
  block_walk_heavy(N, bl, L.bfsh_begin, nheavy, T, S.c[C_NEXT], two);
}

// ---------------------------------------------------------------------------
// Asynchronous global relabel.  The level-synchronous search above pays one
// grid barrier and one dependent load chain per breadth-first level, and the
// reverse searches of a large network are hundreds of levels deep.  Here the
// whole search runs in one phase: a label-correcting search (labels only
// decrease, by atomicMin) driven by a work queue in global memory.  Every
// node whose label drops is queued again, so at the end every label is the
// exact residual distance to the sinks, the same labels the level-by-level
// search sets; the order of work only changes how often a node is expanded.
//
// Queue entries are 64-bit: (label + 1) << 37 | chunk << 27 | node, so an
// entry is never zero and a zero slot is an empty one (the slots used by a
// relabel are cleared by the next one; Lawler ids must stay below 2^27).  A
// node with more than kLightItems arc groups is queued as chunks of at least
// kGqChunk arc groups (at most 1,024 chunks), so one team walks one chunk.
// Teams take slots from gq_head in order, wait for the slot's entry to be
// written, expand it, and count it in gq_done once its own entries are
// queued.  The search is over when gq_done equals gq_tail, read as tail,
// done, tail with acquire loads: an entry is counted done only after the
// entries it produced were counted in the tail, so equal counts mean nothing
// is queued or being expanded.  An entry whose node has a smaller label by
// now is skipped: the entry queued when the label dropped expands it.  A full
// queue sets gq_over; the relabel is then redone level by level.
constexpr unsigned kGqChunk = 16;
static_assert(kLightItems <= (int)kGqChunk, "a light node is queued as one chunk");
constexpr unsigned kGqMaxChunks = 1024;
constexpr unsigned kGqNodeBits = 27;

__device__ __forceinline__ unsigned gq_chunk_size(unsigned items) {
  return items <= kGqChunk * kGqMaxChunks ? kGqChunk : (items + kGqMaxChunks - 1) / kGqMaxChunks;
}

__device__ __forceinline__ unsigned gq_chunks(unsigned items) {
  const unsigned cs = gq_chunk_size(items);
  return items == 0 ? 1u : (items + cs - 1) / cs;
}

__device__ __forceinline__ unsigned long long gq_entry(int z, unsigned chunk, int label) {
  return ((unsigned long long)(label + 1) << 37) | ((unsigned long long)chunk << kGqNodeBits) |
         (unsigned)z;
}

// Queue every chunk of node z (label d, flag byte f) for the lanes with
// `want`.  Warp-collective: one tail atomic per warp; the chunks of large
// nodes are written by the whole warp.
__device__ void gq_push(const NetDev& N, EngineCtl* E, bool want, int z, uint8_t f, int d) {
  const unsigned lane = lane_id();
  unsigned cnt = 0;
  if (want) cnt = (f & kHeavy) ? gq_chunks(node_arcs(N, z).items) : 1u;
  unsigned incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(FULL, incl, o);
    if ((int)lane >= o) incl += t;
  }
  const unsigned total = __shfl_sync(FULL, incl, 31);
  if (total == 0) return;
  unsigned base = 0;
  if (lane == 31) base = atomicAdd(&E->gq_tail, total);
  base = __shfl_sync(FULL, base, 31);
  const unsigned s0 = base + incl - cnt;
  const bool fits = s0 <= N.gq_cap && N.gq_cap - s0 >= cnt;
  if (cnt && !fits) *(volatile unsigned*)&E->gq_over = 1u;
  if (cnt == 1 && fits) st_release_u64(&N.gq[s0], gq_entry(z, 0, d));
  unsigned big = __ballot_sync(FULL, cnt > 1 && fits);
  if (!big) return;
  __syncwarp();   // every lane's label update is ordered before the other lanes' stores
  while (big) {
    const int src = __ffs(big) - 1;
    big &= big - 1;
    const unsigned bs = __shfl_sync(FULL, s0, src), bc = __shfl_sync(FULL, cnt, src);
    const int bz = __shfl_sync(FULL, z, src), bd = __shfl_sync(FULL, d, src);
    for (unsigned c = lane; c < bc; c += 32) st_release_u64(&N.gq[bs + c], gq_entry(bz, c, bd));
  }
}

// Seeding: every sink (the BFS list of ST_GR_INIT, label 0) enters the queue.
__device__ void gr_seed(const NetDev& N, EngineCtl* E, const Sched& L, const Team& T,
                        unsigned lane) {
  const unsigned nl = L.bfs_end, nh = L.bfsh_end, tot = nl + nh;
  const int32_t* bl = N.list[L_BFS];
  for (unsigned i0 = T.tid - lane; i0 < tot; i0 += T.nth) {
    const unsigned i = i0 + lane;
    int y = -1;
    uint8_t f = 0;
    if (i < tot) {
      y = i < nl ? bl[i] : bl[N.NL - 1 - (i - nl)];
      f = N.flags[y];
    }
    gq_push(N, E, y >= 0, y, f, 0);
  }
}

// Label of z lowered to d1 when larger (sources never take labels).  On the
// first label the node's weight joins T_r and, with excess, it joins the
// frontier.  Warp-collective; queues the lanes' lowered nodes.
__device__ __forceinline__ bool gq_relax(const NetDev& N, EngineCtl* E, const Slot& S, int z,
                                         int d1, Acc& a) {
  bool imp = false, first = false;
  uint8_t f = 0;
  if (z >= 0) {
    const int cur = __ldcg(&N.lab0[z]);
    f = N.flags[z];
    if (cur > d1 && !(f & kSource)) {
      const int old = atomicMin(&N.lab0[z], d1);
      if (old > d1) {
        imp = true;
        atomicMin(&N.lab1[z], d1);
        first = old == N.NL;
      }
    }
  }
  gq_push(N, E, imp, z, f, d1);
  bool act = false;
  if (first) {
    if (z < N.n_nodes) a.w += N.node_w[z];
    act = N.excess[z] > 0;
  }
  append_split(act, z, (f & kHeavy) != 0, N.list[L_FRONT], S.act[0], S.act[1], 0, 0, N.NL);
  return imp;
}

// Expand chunk c of node x queued with label d (x < 0: idle team): relax
// every reverse residual arc into x with d + 1.  Skipped when x's label has
// dropped below d since (a later entry of x expands it).
template <int TW>
__device__ void gq_expand(const NetDev& N, EngineCtl* E, const Slot& S, int x, unsigned c, int d,
                          unsigned lane, Acc& a, unsigned& maxd) {
  const unsigned tl = lane & (TW - 1);
  NodeArcs g{0, 0, 0, 0};
  int w = 0, fb = 0;
  unsigned k0 = 0, k1 = 0;
  if (x >= 0) {
    const int cur = __ldcg(&N.lab0[x]);
    g = node_arcs(N, x);
    if (g.kind) {
      w = N.net_w[g.e];
      fb = N.f_b[g.e];
    }
    const unsigned cs = gq_chunk_size(g.items);
    k0 = c * cs;
    k1 = min(k0 + cs, g.items);
    if (cur < d || d >= N.NL) k1 = k0;
  }
  const int d1 = d + 1;
  const unsigned steps = warp_max_u(k1 > k0 ? (k1 - k0 + TW - 1) / TW : 0u);
  for (unsigned st = 0; st < steps; st++) {
    const unsigned k = k0 + st * TW + tl;
    int c1 = -1, c2 = -1;
    if (k < k1) rev_arcs(N, g, k, w, fb, c1, c2, a);
    const bool i1 = gq_relax(N, E, S, c1, d1, a);
    const bool i2 = gq_relax(N, E, S, c2, d1, a);
    if (i1 || i2) maxd = max(maxd, (unsigned)d1);
  }
}

// The search itself: warps below P.gr_warps of every CTA serve the queue,
// four 8-lane teams per warp, until it is finished, overflowed, or an error
// or the time bound stops it.
__device__ void gr_run(const NetDev& N, EngineCtl* E, const Sched& L, const Slot& S,
                       unsigned lane, Acc& a, const Params& P) {
  if ((threadIdx.x >> 5) >= P.gr_warps) return;
  constexpr unsigned NONE = 0xffffffffu;
  const unsigned tl = lane & (kTeam - 1), lead = lane & ~(unsigned)(kTeam - 1);
  unsigned slot = NONE, maxd = 0, idle = 0;
  unsigned long long t0 = 0;
  for (;;) {
    // slots for the teams that have none: one atomic per warp
    const unsigned m = __ballot_sync(FULL, slot == NONE && tl == 0);
    if (m) {
      const int ld = __ffs(m) - 1;
      unsigned base = 0;
      if ((int)lane == ld) base = atomicAdd(&E->gq_head, (unsigned)__popc(m));
      base = __shfl_sync(FULL, base, ld);
      if (slot == NONE) slot = base + __popc(m & ((1u << lead) - 1u));
    }
    unsigned long long ent = 0;
    if (tl == 0 && slot < N.gq_cap) ent = ld_acquire_u64(&N.gq[slot]);
    ent = __shfl_sync(FULL, ent, lead);
    const bool ready = ent != 0ull;
    const unsigned rm = __ballot_sync(FULL, ready);
    if (rm) {
      const int x = ready ? (int)(ent & ((1u << kGqNodeBits) - 1u)) : -1;
      const unsigned c = ready ? (unsigned)(ent >> kGqNodeBits) & (kGqMaxChunks - 1u) : 0u;
      const int d = ready ? (int)(ent >> 37) - 1 : 0;
      gq_expand<kTeam>(N, E, S, x, c, d, lane, a, maxd);
      if (ready) slot = NONE;
      __syncwarp();
      if (lane == 0) red_release_add(&E->gq_done, (unsigned)__popc(rm) / kTeam);
      idle = 0;
      t0 = 0;
      continue;
    }
    if ((++idle & 7u) == 0) {
      int stop = 0;
      if (lane == 0) {
        if (ld_volatile_int((const int*)&E->gq_over) || ld_volatile_int(&E->c.err) != kDevOk) {
          stop = 1;
        } else {
          const unsigned t1 = ld_acquire(&E->gq_tail);
          const unsigned dn = ld_acquire(&E->gq_done);
          const unsigned t2 = ld_acquire(&E->gq_tail);
          if (dn == t1 && t1 == t2) {
            stop = 1;
          } else {
            const unsigned long long t = globaltimer();
            if (t0 == 0) {
              t0 = t;
            } else if (t - t0 > P.timeout_ns) {
              atomicCAS(&E->c.err, kDevOk, kDevTimeout);
              E->c.err_where = 3;
              stop = 1;
            }
          }
        }
      }
      if (__shfl_sync(FULL, stop, 0)) break;
    }
    if (idle > 32) __nanosleep(64);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) maxd = max(maxd, __shfl_xor_sync(FULL, maxd, o));
  if (lane == 0 && maxd) atomicMax(&E->gq_maxd, maxd);
}

// Source-side cut, step 1: seeds are the sources and every non-sink node with
// positive excess (Section 8.4, "Source-Side Cut").
__device__ void sr_init(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                        unsigned lane, Acc& a) {
  for (unsigned x0 = T.tid - lane; x0 < (unsigned)N.NL; x0 += T.nth) {
    const unsigned x = x0 + lane;
    bool seed = false, hv = false, expand = false;
    if (x < (unsigned)N.NL) {
      const uint8_t f = N.flags[x];
      hv = (f & kHeavy) != 0;
      const bool src = (f & kSource) != 0;
      seed = src || (!(f & kSink) && N.excess[x] > 0);
      N.insr[x] = seed ? 1 : 0;
      if (seed) {
        N.stamp[x] = L.epoch;
        if (x < (unsigned)N.n_nodes) a.w += N.node_w[x];
      }
      expand = seed && (!src || L.sr_one == 0 || (int)x == L.sr_one - 1);
    }
    append_split(expand, (int)x, hv, N.list[L_BFS], S.c[C_BFS], S.c[C_BFSH], 0, 0, N.NL);
  }
}

// Source-side cut after adding one source u whose arcs were left as they
// were (a piercing node without augmenting path): the preflow is still a
// maximum preflow, S_r only grows by what u reaches, so the search starts at
// u alone and keeps every node already in S_r.
__device__ void sr_add(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                       unsigned lane, Acc& a) {
  if (T.tid >= 32) return;
  const int u = L.seed;
  bool seed = false, hv = false;
  if (lane == 0 && u >= 0 && !N.insr[u]) {
    N.insr[u] = 1;
    N.stamp[u] = L.epoch;
    hv = (N.flags[u] & kHeavy) != 0;
    if (u < N.n_nodes) a.w += N.node_w[u];
    seed = true;
  }
  append_split(seed, u, hv, N.list[L_BFS], S.c[C_BFS], S.c[C_BFSH], 0, 0, N.NL);
}

// Forward residual arcs out of x with (u, e_in) uncapped, arc group k.
__device__ __forceinline__ void fwd_arcs(const NetDev& N, const NodeArcs& g, unsigned k, int w,
                                         int fb, int& c1, int& c2, Acc& a) {
  const int nh = N.n_nodes, m = N.m_nets;
  c1 = c2 = -1;
  if (g.kind == 0) {
    // out of a hypernode: (u, e_in) always, (u, e_out) when f_out > 0
    const int2 it = N.inc[g.beg + k];
    c1 = nh + it.x;
    if (N.f_out[it.y] > 0) c2 = nh + m + it.x;
    a.hyper++;
  } else if (k == 0) {
    // out of e_in: bridge when f_b < w; out of e_out: (e_out, e_in) when f_b > 0
    if (g.kind == 1) {
      if (fb < w) c1 = nh + m + g.e;
    } else if (fb > 0) {
      c1 = nh + g.e;
    }
  } else {
    // out of e_in: (e_in, u) when f_in > 0; out of e_out: (e_out, u) always
    const unsigned p = g.beg + k - 1;
    if (g.kind == 2 || N.f_in[p] > 0) c1 = N.pin[p];
    a.net++;
  }
}

// The heads c[0 .. K) of K arc groups (-1: none; a node may appear twice)
// that are not yet in S_r join it: the stamp exchange of the search's epoch
// decides which visit wins.  The loads of all K are issued first, and the
// appends go in ballot passes of two per lane.
template <int K>
__device__ __forceinline__ void sr_emit(const NetDev& N, const Sched& L, const Slot& S,
                                        const int (&c)[K], Acc& a) {
  uint8_t in[K], f[K];
  bool k[K];
#pragma unroll
  for (int i = 0; i < K; i++) {
    in[i] = 1;
    f[i] = 0;
    if (c[i] >= 0) {
      in[i] = N.insr[c[i]];
      f[i] = N.flags[c[i]];
    }
  }
#pragma unroll
  for (int i = 0; i < K; i++) {
    k[i] = !in[i];
    if (k[i]) k[i] = atomicExch(&N.stamp[c[i]], L.epoch) != L.epoch;
  }
#pragma unroll
  for (int i = 0; i < K; i++)
    if (k[i]) {
      N.insr[c[i]] = 1;
      if (c[i] < N.n_nodes) a.w += N.node_w[c[i]];
    }
#pragma unroll
  for (int i = 0; i < K; i += 2)
    append_split2(k[i], c[i], (f[i] & kHeavy) != 0, k[i + 1], c[i + 1], (f[i + 1] & kHeavy) != 0,
                  N.list[L_BFS], S.c[C_BFS], S.c[C_BFSH], L.bfs_end, L.bfsh_end, N.NL);
}

// Source-side cut, one level: forward BFS over residual arcs with (u, e_in)
// uncapped.  Light nodes by level_light, heavy ones by block_walk_heavy.
__device__ void sr_level(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                         unsigned lane, Acc& a) {
  const int32_t* bl = N.list[L_BFS];
  const unsigned nlight = L.bfs_end - L.bfs_begin, nheavy = L.bfsh_end - L.bfsh_begin;
  auto one = [&](const NodeArcs& g, unsigned k, int w, int fb) {
    int c[2] = {-1, -1};
    if (k != kNoArc) fwd_arcs(N, g, k, w, fb, c[0], c[1], a);
    sr_emit<2>(N, L, S, c, a);
  };
  auto two = [&](const WalkArc& A, const WalkArc& B) {
    int c[4] = {-1, -1, -1, -1};
    if (A.k != kNoArc) fwd_arcs(N, A.g, A.k, A.w, A.fb, c[0], c[1], a);
    if (B.k != kNoArc) fwd_arcs(N, B.g, B.k, B.w, B.fb, c[2], c[3], a);
    sr_emit<4>(N, L, S, c, a);
  };
  level_light(N, bl + L.bfs_begin, nlight, T, lane, S.c[C_RELAB], one, two);
  block_walk_heavy(N, bl, L.bfsh_begin, nheavy, T, S.c[C_NEXT], two);
}

// Distance from the original cut (reading of Section 6 "Region Growing" and
// Section 7 "Piercing"): breadth-first search inside the region from the
// vertices at distance 1, a warp per vertex (light part of the BFS list
// only).  Level i holds the vertices at distance i + 1.
__device__ void dist_init(const NetDev& N, const Team& T, const Slot& S, unsigned lane) {
  for (unsigned u0 = T.tid - lane; u0 < (unsigned)N.n_nodes; u0 += T.nth) {
    const unsigned u = u0 + lane;
    const bool seed = u >= 2 && u < (unsigned)N.n_nodes && N.node_dist[u] == 1;
    append_plain(seed, (int)u, N.list[L_BFS], S.c[C_BFS], 0);
  }
}

__device__ void dist_level(const NetDev& N, const Sched& L, const Team& T, const Slot& S,
                           unsigned lane) {
  const int d2 = L.level + 2;
  int32_t* bl = N.list[L_BFS];
  for (unsigned w = L.bfs_begin + T.gwarp; w < L.bfs_end; w += T.nwarps) {
    const int u = bl[w];
    for (unsigned j = N.node_off[u]; j < N.node_off[u + 1]; j++) {
      const int e = N.inc[j].x;
      const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
      for (unsigned p0 = beg; p0 < end; p0 += 32) {
        const unsigned p = p0 + lane;
        bool claim = false;
        int v = -1;
        if (p < end) {
          v = N.pin[p];
          if (v >= 2 && N.node_dist[v] < 0)
            claim = atomicCAS(&N.node_dist[v], -1, min(d2, kDistFar)) == -1;
        }
        append_plain(claim, v, bl, S.c[C_BFS], L.bfs_end);
      }
    }
  }
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ Slot slot_of(EngineCtl* E, unsigned k) {
  const unsigned sl = k % 3;
  Slot S;
#pragma unroll
  for (int i = 0; i < C_COUNT; i++) S.c[i] = &E->cnt3[i][sl];
  S.flow = &E->flow3[sl];
  S.act[0] = &E->gr_act[0];
  S.act[1] = &E->gr_act[1];
  return S;
}

// One phase of the current state by team T with counters S; hypernode
// weights reached go to w_sh.
__device__ void run_phase_s(const NetDev& N, EngineCtl* E, const Sched& L, const Team& T,
                            const Slot& S, unsigned lane, Acc& a, long long* w_sh,
                            const Params& P) {
  switch (L.state) {
    case ST_ROUND_A: phase_a(N, L, T, S, lane, a, E); break;
    case ST_ROUND: phase_round(N, L, T, S, lane, a, P); break;
    case ST_FLUSH: phase_flush(N, L, T); break;
    case ST_ROUND_B: phase_b(N, L, T, S, lane, a); break;
    case ST_GR_INIT: gr_init(N, E, L, T, S, lane, a); break;
    case ST_GR_SEED: gr_seed(N, E, L, T, lane); break;
    case ST_GR_RUN: gr_run(N, E, L, S, lane, a, P); break;
    case ST_GR_ADD: gr_add(N, L, T, S, lane, a); break;
    case ST_GR_LEVEL: gr_level(N, E, L, T, S, lane, a); break;
    case ST_SR_INIT: sr_init(N, L, T, S, lane, a); break;
    case ST_SR_ADD: sr_add(N, L, T, S, lane, a); break;
    case ST_SR_LEVEL: sr_level(N, L, T, S, lane, a); break;
    case ST_DIST_INIT: dist_init(N, T, S, lane); break;
    case ST_DIST_LEVEL: dist_level(N, L, T, S, lane); break;
    default: break;
  }
  if (a.w) {
    atomicAdd((unsigned long long*)w_sh, (unsigned long long)a.w);
    a.w = 0;
  }
}

// One grid phase: counters in the phase's slot of the control block.
__device__ void run_phase(const NetDev& N, EngineCtl* E, const Sched& L, const Team& T,
                          unsigned lane, Acc& a, long long* w_sh, const Params& P) {
  run_phase_s(N, E, L, T, slot_of(E, L.phase), lane, a, w_sh, P);
}

__device__ __forceinline__ void flush_weight(EngineCtl* E, unsigned k, long long* w_sh) {
  if (*w_sh) {
    atomicAdd((unsigned long long*)&E->w3[k % 3], (unsigned long long)*w_sh);
    *w_sh = 0;
  }
}

// Per-state device time, kept by thread 0 of CTA 0.
struct Clock {
  unsigned long long t_last;
  unsigned long long ns[10], cnt[10];
};

// Returns the device time of the phase that just ended.
__device__ __forceinline__ unsigned long long tick(Clock& ck, int st) {
  const unsigned long long t = globaltimer();
  const unsigned long long dt = t - ck.t_last;
  st = st < 10 ? st : 9;
  ck.ns[st] += dt;
  ck.cnt[st]++;
  ck.t_last = t;
  return dt;
}

// Phase trace (when enabled): four words per phase,
//   (state | solo << 5) << 58 | light input << 29 | heavy input,
//   light output << 32 | heavy output, flow value, device time (ns).
// Inputs are the frontier (push), the next list (relabel/apply) or the BFS
// level; outputs the list the phase appended to.  Counts are clipped to 29 /
// 32 bits.
__device__ void trace_phase(const NetDev& N, Ctl* c, const Sched& L, int st, bool solo,
                            const Snap& q, unsigned long long dt) {
  if (!N.trace || c->trace_len >= N.trace_cap) return;
  unsigned long long a = 0, b = 0, oa = 0, ob = 0;
  if (st == ST_ROUND_A || st == ST_ROUND || st == ST_FLUSH) {
    a = L.fcnt; b = L.fcnth; oa = q.c[C_NEXT]; ob = q.c[C_NEXTH];
  } else if (st == ST_ROUND_B) {
    a = L.ncnt; b = L.ncnth; oa = q.c[C_FRONT]; ob = q.c[C_FRONTH];
  } else {
    a = L.bfs_end - L.bfs_begin; b = L.bfsh_end - L.bfsh_begin;
    oa = q.c[C_BFS]; ob = q.c[C_BFSH];
  }
  const unsigned long long m29 = (1ull << 29) - 1;
  unsigned long long* w = N.trace + 4 * c->trace_len;
  w[0] = ((unsigned long long)((st & 31) | (solo ? 32 : 0)) << 58) | (min(a, m29) << 29) |
         min(b, m29);
  w[1] = (min(oa, 0xffffffffull) << 32) | min(ob, 0xffffffffull);
  w[2] = L.flow;
  w[3] = dt;
  c->trace_len++;
}

__device__ __forceinline__ bool is_level(int st) {
  return st == ST_GR_LEVEL || st == ST_SR_LEVEL || st == ST_DIST_LEVEL;
}

// Work of the next BFS level: light nodes, plus heavy ones counted 32 times
// (a CTA walks a heavy node's arcs alone).
__device__ __forceinline__ unsigned level_size(const Sched& L) {
  return (L.bfs_end - L.bfs_begin) + 32u * (L.bfsh_end - L.bfsh_begin);
}

// Whether the next phase runs CTA-alone: small frontiers (the ST_TAIL state
// that advance() picks) and thin breadth-first-search levels.  Every CTA
// evaluates it on its identical copy of the state.
__device__ __forceinline__ bool solo_next(const Sched& L, const Params& P) {
  return L.state == ST_TAIL || (is_level(L.state) && level_size(L) <= P.bfs_enter);
}

// Phases run by one CTA while the work stays small: rounds while the
// frontier has at most tail_exit nodes, breadth-first-search levels while
// they have at most bfs_exit nodes.  Block barriers instead of grid barriers
// and append counters in shared memory, so a phase costs its own dependent
// loads and nothing else.  The active-node counters of a running global
// relabel move into shared memory and back; on leaving, every phase slot of
// the control block is zeroed (the other CTAs wait at the grid barrier).
// Leaves with L holding the next grid state.
__device__ void solo_phases(const NetDev& N, EngineCtl* E, const Params& P, Sched& L,
                            unsigned lane, Acc& a, long long* w_sh, Clock& ck, SoloSh& sh) {
  const Team T{threadIdx.x >> 5, blockDim.x >> 5, threadIdx.x, blockDim.x, 0, 1};
  __syncthreads();   // every thread has read the caller's state before it is rewritten
  if (threadIdx.x == 0) {
    if (L.state == ST_TAIL) L.state = round_state(P);
    sh.act[0] = ld_cg(&E->gr_act[0]);
    sh.act[1] = ld_cg(&E->gr_act[1]);
  }
  Slot S;
  for (int i = 0; i < C_COUNT; i++) S.c[i] = &sh.c[i];
  S.flow = &sh.flow;
  S.act[0] = &sh.act[0];
  S.act[1] = &sh.act[1];
  const unsigned long long t0 = globaltimer();
  for (;;) {
    if (threadIdx.x == 0) {
      for (int i = 0; i < C_COUNT; i++) sh.c[i] = 0;
      sh.flow = 0;
    }
    __syncthreads();
    run_phase_s(N, E, L, T, S, lane, a, w_sh, P);
    __syncthreads();
    if (threadIdx.x == 0) {
      Snap q;
      for (int i = 0; i < C_COUNT; i++) q.c[i] = sh.c[i];
      q.act = sh.act[0];
      q.acth = sh.act[1];
      q.flow = sh.flow;
      q.w = *w_sh;
      *w_sh = 0;
      q.key = 0;
      q.node = -1;
      const unsigned long long dt = tick(ck, ST_TAIL);
      const int s1 = L.state;
      trace_phase(N, &E->c, L, s1, true, q, dt);
      advance(L, q, P, N, &E->c);
      L.phase++;
      const int s2 = L.state;
      bool stay;
      if (is_level(s1) && !is_level(s2)) {
        // a search ended: labels claimed by atomics must reach the plain
        // loads of the next phases, which the grid barrier's acquire does
        stay = false;
      } else if (s2 == ST_TAIL) {
        L.state = round_state(P);
        stay = true;
      } else if (s2 == ST_ROUND_B || s2 == ST_FLUSH) {
        stay = true;
      } else if (s2 == ST_ROUND_A || s2 == ST_ROUND) {
        stay = L.fcnt + L.fcnth <= P.tail_exit;
      } else if (is_level(s2)) {
        stay = level_size(L) <= P.bfs_exit;
      } else {
        stay = false;
      }
      if (stay && (ld_volatile_int(&E->c.err) != kDevOk || globaltimer() - t0 > P.timeout_ns)) {
        // bounded like a grid barrier wait: give up with an error status
        atomicCAS(&E->c.err, kDevOk, kDevTimeout);
        E->c.err_where = 2;
        L.state = ST_DONE;
        stay = false;
      }
      sh.stay = stay ? 1 : 0;
    }
    __syncthreads();
    if (!sh.stay) break;
  }
  __syncthreads();   // every thread has read sh.stay
  if (threadIdx.x == 0) {
    E->gr_act[0] = sh.act[0];
    E->gr_act[1] = sh.act[1];
    for (unsigned sl = 0; sl < 3; sl++) clear_slot(E, sl, false);
    __threadfence();
  }
  __syncthreads();
}

__device__ void load_sched(Sched& L, const EngineCtl* E) {
  const volatile Sched* v = &E->s;
  L.state = v->state;
  L.lp = v->lp;
  L.fcnt = v->fcnt;
  L.fcnth = v->fcnth;
  L.ncnt = v->ncnt;
  L.ncnth = v->ncnth;
  L.rcnt = v->rcnt;
  L.bfs_begin = v->bfs_begin;
  L.bfs_end = v->bfs_end;
  L.bfsh_begin = v->bfsh_begin;
  L.bfsh_end = v->bfsh_end;
  L.level = v->level;
  L.epoch = v->epoch;
  L.after_gr_exit = v->after_gr_exit;
  L.phase = v->phase;
  L.seed = v->seed;
  L.last_gr = v->last_gr;
  L.gr_sync = v->gr_sync;
  L.gr_one = v->gr_one;
  L.sr_one = v->sr_one;
  L.fsel = v->fsel;
  L.rounds = v->rounds;
  L.grs = v->grs;
  L.gr_levels = v->gr_levels;
  L.gq_items = v->gq_items;
  L.gq_prev = v->gq_prev;
  L.gq_overs = v->gq_overs;
  L.work = v->work;
  L.stall = v->stall;
  L.flow = v->flow;
  L.flow_ref = v->flow_ref;
  L.wS = v->wS;
  L.wT = v->wT;
  L.wS_set = v->wS_set;
  L.wT_set = v->wT_set;
}

__device__ void store_sched(EngineCtl* E, const Sched& L) {
  volatile Sched* v = &E->s;
  v->state = L.state;
  v->lp = L.lp;
  v->fcnt = L.fcnt;
  v->fcnth = L.fcnth;
  v->ncnt = L.ncnt;
  v->ncnth = L.ncnth;
  v->rcnt = L.rcnt;
  v->bfs_begin = L.bfs_begin;
  v->bfs_end = L.bfs_end;
  v->bfsh_begin = L.bfsh_begin;
  v->bfsh_end = L.bfsh_end;
  v->level = L.level;
  v->epoch = L.epoch;
  v->after_gr_exit = L.after_gr_exit;
  v->phase = L.phase;
  v->seed = L.seed;
  v->last_gr = L.last_gr;
  v->gr_sync = L.gr_sync;
  v->gr_one = L.gr_one;
  v->sr_one = L.sr_one;
  v->fsel = L.fsel;
  v->rounds = L.rounds;
  v->grs = L.grs;
  v->gr_levels = L.gr_levels;
  v->gq_items = L.gq_items;
  v->gq_prev = L.gq_prev;
  v->gq_overs = L.gq_overs;
  v->work = L.work;
  v->stall = L.stall;
  v->flow = L.flow;
  v->flow_ref = L.flow_ref;
  v->wS = L.wS;
  v->wT = L.wT;
  v->wS_set = L.wS_set;
  v->wT_set = L.wT_set;
}

__global__ void __launch_bounds__(kEngineThreads) engine_kernel(NetDev N, EngineCtl* E, Params P) {
  __shared__ Sched L;
  __shared__ Acc acc_sh;
  __shared__ long long w_sh;
  __shared__ Clock ck;
  __shared__ SoloSh solo;
  const unsigned lane = lane_id();
  const unsigned wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const Team G{blockIdx.x * nwb + wib, gridDim.x * nwb, blockIdx.x * blockDim.x + threadIdx.x,
               gridDim.x * blockDim.x, blockIdx.x, gridDim.x};
  const bool cta0 = blockIdx.x == 0;
  if (threadIdx.x == 0) {
    load_sched(L, E);
    if (ld_volatile_int(&E->c.err) != kDevOk) L.state = ST_DONE;   // left by an earlier launch
    if (L.state == ST_ROUND_A && P.fused_rounds) {
      // rounds set up by the host (new excess in the frontier list)
      L.state = ST_ROUND;
      L.fsel = L_FRONT;
    }
    L.flow = *(const volatile unsigned long long*)&E->c.flow;  // host kernels add to it
    acc_sh = Acc{0, 0, 0, 0, 0};
    w_sh = 0;
    for (int i = 0; i < 10; i++) ck.ns[i] = ck.cnt[i] = 0;
    ck.t_last = globaltimer();
  }
  __syncthreads();
  Acc a{0, 0, 0, 0, 0};
  unsigned bar_seq = 0;
  for (;;) {
    const int st = L.state;
    if (st == ST_DONE) break;
    if (solo_next(L, P)) {
      if (cta0) {
        solo_phases(N, E, P, L, lane, a, &w_sh, ck, solo);
        if (threadIdx.x == 0) store_sched(E, L);
      }
      const bool ok = grid_barrier(E, gridDim.x * ++bar_seq, P.timeout_ns);
      if (threadIdx.x == 0) {
        if (!cta0) load_sched(L, E);
        if (!ok) L.state = ST_DONE;
      }
      __syncthreads();
      continue;
    }
    if (cta0 && threadIdx.x == 0)
      clear_slot(E, (L.phase + 1) % 3, st == ST_GR_INIT || st == ST_GR_ADD);
    run_phase(N, E, L, G, lane, a, &w_sh, P);
    __syncthreads();
    if (threadIdx.x == 0) flush_weight(E, L.phase, &w_sh);
    const bool ok = grid_barrier(E, gridDim.x * ++bar_seq, P.timeout_ns);
    if (threadIdx.x == 0) {
      if (!ok) {
        L.state = ST_DONE;
      } else {
        const Snap q = take_snap(E, L.phase);
        if (cta0) trace_phase(N, &E->c, L, st, false, q, tick(ck, st));
        advance(L, q, P, N, &E->c);
        L.phase++;
      }
    }
    __syncthreads();
  }
  // statistics and the published state (CTA 0)
  if (a.hyper) atomicAdd(&acc_sh.hyper, a.hyper);
  if (a.net) atomicAdd(&acc_sh.net, a.net);
  if (a.nodes) atomicAdd(&acc_sh.nodes, a.nodes);
  if (a.pushes) atomicAdd(&acc_sh.pushes, a.pushes);
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&E->c.items_hyper, acc_sh.hyper);
    atomicAdd(&E->c.items_net, acc_sh.net);
    atomicAdd(&E->c.node_visits, acc_sh.nodes);
    atomicAdd(&E->c.pushes, acc_sh.pushes);
    if (cta0) {
      store_sched(E, L);
      E->c.flow = L.flow;
      E->c.rounds = L.rounds;
      E->c.global_relabels = L.grs;
      E->c.gr_levels = L.gr_levels;
      E->c.gq_items = L.gq_items;
      E->c.gq_overs = L.gq_overs;
      if (L.wS_set) E->c.wS = L.wS;
      if (L.wT_set) E->c.wT = L.wT;
      for (int i = 0; i < 10; i++) {
        E->c.state_ns[i] += ck.ns[i];
        E->c.state_cnt[i] += ck.cnt[i];
      }
    }
  }
}

#include "engine_batch.cuh"

}  // namespace hfp
