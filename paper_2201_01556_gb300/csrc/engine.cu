// Persistent flow engine: synchronous push-relabel on the Lawler expansion,
// simulated directly on the flow hypergraph, with global relabeling and the
// residual BFS of the source-side cut.  One cooperative launch runs the whole
// loop; every grid barrier ends with a serial section (run by the last CTA to
// arrive) that snapshots the list counters and picks the next state.
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
// Difference from the paper's round: a round here is split into a push phase
// and a relabel phase separated by a grid barrier.  Pushes use only the old
// labels, and a node relabels (against the old labels of its neighbours, read
// from the other buffer of a double-buffered label array) only after every
// push of the round has landed, so the new residual arcs created by
// concurrent pushes are always seen.  Labels therefore stay valid at all
// times, the push-relabel conflict of Section 8.2 cannot occur, and no
// winning criterion is needed: an arc can only be admissible in one
// direction under one labelling.  The run is deterministic.
#include "kernels.cuh"

namespace hfp {

constexpr unsigned FULL = 0xffffffffu;

struct Acc {
  long long w;                 // hypernode weight found in this phase
  unsigned long long hyper, net, nodes, pushes;
};

__device__ __forceinline__ int32_t* lab_cur(const NetDev& N, int lp) { return lp ? N.lab1 : N.lab0; }

// ---------------------------------------------------------------------------
// serial section: runs in exactly one thread while the rest of the grid waits
__device__ void begin_gr(EngineCtl* E, int final_gr) {
  E->c.global_relabels++;
  E->s.state = ST_GR_INIT;
  E->s.final_gr = final_gr;
  E->cnt[L_BFS] = 0;
  E->cnt[L_FRONT] = 0;
  E->c.wT = 0;
}

__device__ void control(EngineCtl* E, const NetDev& N, const Params& P) {
  Sched& s = E->s;
  Ctl& c = E->c;
  switch (s.state) {
    case ST_ROUND_A:
      s.ncnt = E->cnt[L_NEXT];
      E->cnt[L_NEXT] = 0;
      s.state = ST_ROUND_B;
      break;
    case ST_ROUND_B: {
      c.rounds++;
      c.work_since_gr += (unsigned long long)s.fcnt + s.ncnt;
      s.fcnt = E->cnt[L_FRONT];
      E->cnt[L_FRONT] = 0;
      s.rcnt = E->cnt[L_RELAB];
      E->cnt[L_RELAB] = 0;
      s.lp ^= 1;
      s.epoch++;
      if (c.flow != E->round_flow_ref || s.fcnt >= P.stall_nodes) {
        E->round_flow_ref = c.flow;
        c.stall_rounds = 0;
      } else {
        c.stall_rounds++;
      }
      if (s.fcnt == 0) {
        begin_gr(E, 1);
      } else if (c.rounds >= P.max_rounds) {
        c.err = kDevIterLimit;
        s.state = ST_DONE;
      } else if (c.work_since_gr >= P.gr_work || c.stall_rounds >= P.stall_rounds) {
        begin_gr(E, 0);
      } else {
        s.state = ST_ROUND_A;
      }
      break;
    }
    case ST_GR_INIT:
      s.bfs_begin = 0;
      s.bfs_end = E->cnt[L_BFS];
      s.level = 0;
      s.state = ST_GR_LEVEL;
      break;
    case ST_GR_LEVEL: {
      unsigned e = E->cnt[L_BFS];
      c.gr_levels++;
      if (e == s.bfs_end) {
        E->cnt[L_BFS] = 0;
        s.fcnt = E->cnt[L_FRONT];
        E->cnt[L_FRONT] = 0;
        s.rcnt = 0;
        E->cnt[L_RELAB] = 0;
        E->cnt[L_NEXT] = 0;
        s.lp = 0;
        s.epoch++;
        c.work_since_gr = 0;
        c.stall_rounds = 0;
        E->round_flow_ref = c.flow;
        s.state = (s.fcnt == 0 || s.after_gr_exit) ? ST_DONE : ST_ROUND_A;
      } else {
        s.bfs_begin = s.bfs_end;
        s.bfs_end = e;
        s.level++;
      }
      break;
    }
    case ST_SR_INIT:
      s.bfs_begin = 0;
      s.bfs_end = E->cnt[L_BFS];
      s.level = 0;
      s.state = ST_SR_LEVEL;
      break;
    case ST_SR_LEVEL: {
      unsigned e = E->cnt[L_BFS];
      if (e == s.bfs_end) {
        E->cnt[L_BFS] = 0;
        s.epoch++;
        s.state = ST_DONE;
      } else {
        s.bfs_begin = s.bfs_end;
        s.bfs_end = e;
        s.level++;
      }
      break;
    }
    case ST_DIST_INIT:
      s.bfs_begin = 0;
      s.bfs_end = E->cnt[L_BFS];
      s.level = 0;
      s.state = ST_DIST_LEVEL;
      break;
    case ST_DIST_LEVEL: {
      unsigned e = E->cnt[L_BFS];
      if (e == s.bfs_end) {
        E->cnt[L_BFS] = 0;
        s.state = ST_DONE;
      } else {
        s.bfs_begin = s.bfs_end;
        s.bfs_end = e;
        s.level++;
      }
      break;
    }
    default:
      s.state = ST_DONE;
  }
}

// Grid barrier with a serial section.  The wait is bounded by P.timeout_ns of
// globaltimer; on expiry ctl->err is set and every CTA leaves the loop.
__device__ bool grid_step(EngineCtl* E, const NetDev& N, const Params& P, Sched* ss,
                          bool transition, Acc* acc_sh, int acc_target) {
  __syncthreads();
  if (threadIdx.x == 0) {
    if (acc_target == 1 && acc_sh->w) atomicAdd((unsigned long long*)&E->c.wS, (unsigned long long)acc_sh->w);
    if (acc_target == 2 && acc_sh->w) atomicAdd((unsigned long long*)&E->c.wT, (unsigned long long)acc_sh->w);
    acc_sh->w = 0;
    unsigned nb = gridDim.x;
    unsigned gen = ld_acquire(&E->c.bar_gen);
    __threadfence();
    unsigned arrived = atomicAdd(&E->c.bar_count, 1u);
    if (arrived == nb - 1) {
      __threadfence();
      if (transition && ld_volatile_int(&E->c.err) == kDevOk) control(E, N, P);
      if (ld_volatile_int(&E->c.err) != kDevOk) E->s.state = ST_DONE;
      atomicExch(&E->c.bar_count, 0u);
      __threadfence();
      st_release(&E->c.bar_gen, gen + 1);
    } else {
      unsigned long long t0 = globaltimer();
      unsigned spins = 0;
      while (ld_acquire(&E->c.bar_gen) == gen) {
        if (ld_volatile_int(&E->c.err) != kDevOk) break;
        if ((++spins & 63u) == 0 && globaltimer() - t0 > P.timeout_ns) {
          atomicCAS(&E->c.err, kDevOk, kDevTimeout);
          E->c.err_where = 1;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    const volatile Sched* vs = &E->s;
    ss->state = vs->state;
    ss->lp = vs->lp;
    ss->fcnt = vs->fcnt;
    ss->ncnt = vs->ncnt;
    ss->rcnt = vs->rcnt;
    ss->bfs_begin = vs->bfs_begin;
    ss->bfs_end = vs->bfs_end;
    ss->level = vs->level;
    ss->epoch = vs->epoch;
    if (ld_volatile_int(&E->c.err) != kDevOk) ss->state = ST_DONE;
  }
  __syncthreads();
  return ss->state != ST_DONE;
}

// ---------------------------------------------------------------------------
// push delivery: returns true when y must be appended to the next list
__device__ __forceinline__ bool deliver(const NetDev& N, int y, long long d, unsigned epoch,
                                        long long& sink_acc) {
  uint8_t fl = N.flags[y];
  if (fl & kSink) {
    sink_acc += d;
    return false;
  }
  if (fl & kSource) return false;
  atomicAdd((unsigned long long*)&N.delta[y], (unsigned long long)d);
  return atomicExch(&N.stamp[y], epoch) != epoch;
}

// Discharge of one node by one warp (Section 8.1, one scan of its residual
// arcs; pushes go on admissible arcs in arc order until the excess is gone).
__device__ void discharge(const NetDev& N, EngineCtl* E, int x, const int32_t* Lr,
                          unsigned epoch, unsigned lane, long long& sink_acc, Acc& a) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  const long long ex = N.excess[x];
  const int dx = Lr[x];
  if (ex <= 0 || dx >= NL) return;
  const int dt = dx - 1;
  long long rem = ex;
  int32_t* nextl = N.list[L_NEXT];
  unsigned* ncnt = &E->cnt[L_NEXT];
  if (x < nh) {
    // hypernode: arcs (u, e_in) with residual w(e) - f_in, (u, e_out) with f_out
    const unsigned beg = N.node_off[x], end = N.node_off[x + 1];
    for (unsigned j0 = beg; j0 < end; j0 += 32) {
      const unsigned j = j0 + lane;
      long long r1 = 0, r2 = 0;
      int e = 0, p = 0, fi = 0, fo = 0;
      if (j < end) {
        int2 it = N.inc[j];
        e = it.x;
        p = it.y;
        int w = N.net_w[e];
        fi = N.f_in[p];
        fo = N.f_out[p];
        if (w > fi && Lr[nh + e] == dt) r1 = w - fi;
        if (fo > 0 && Lr[nh + m + e] == dt) r2 = fo;
      }
      const long long r = r1 + r2;
      const long long incl = warp_incl_scan(r);
      const long long take = min(max(rem - (incl - r), 0LL), r);
      const long long t1 = min(take, r1), t2 = take - t1;
      bool a1 = false, a2 = false;
      if (t1 > 0) {
        N.f_in[p] = fi + (int)t1;
        a1 = deliver(N, nh + e, t1, epoch, sink_acc);
      }
      if (t2 > 0) {
        N.f_out[p] = fo - (int)t2;
        a2 = deliver(N, nh + m + e, t2, epoch, sink_acc);
      }
      a.pushes += (t1 > 0) + (t2 > 0);
      warp_append(a1, nh + e, nextl, ncnt);
      warp_append(a2, nh + m + e, nextl, ncnt);
      a.hyper += (j < end);
      const long long tot = __shfl_sync(FULL, incl, 31);
      rem -= min(rem, tot);
      if (rem == 0) break;
    }
  } else if (x < nh + m) {
    // in-node: bridge (e_in, e_out) with residual w - f_b; (e_in, u) with f_in
    const int e = x - nh;
    const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
    const int w = N.net_w[e], fb = N.f_b[e], eout = nh + m + e;
    const unsigned items = 1 + (end - beg);
    for (unsigned i0 = 0; i0 < items; i0 += 32) {
      const unsigned i = i0 + lane;
      long long r = 0;
      int y = -1, fi = 0;
      unsigned p = 0;
      if (i == 0) {
        if (w > fb && Lr[eout] == dt) { r = w - fb; y = eout; }
      } else if (i < items) {
        p = beg + i - 1;
        fi = N.f_in[p];
        if (fi > 0) {
          int u = N.pin[p];
          if (Lr[u] == dt) { r = fi; y = u; }
        }
      }
      const long long incl = warp_incl_scan(r);
      const long long take = min(max(rem - (incl - r), 0LL), r);
      bool ap = false;
      if (take > 0) {
        if (i == 0) N.f_b[e] = fb + (int)take;
        else N.f_in[p] = fi - (int)take;
        ap = deliver(N, y, take, epoch, sink_acc);
        a.pushes++;
      }
      warp_append(ap, y, nextl, ncnt);
      a.net += (i < items);
      const long long tot = __shfl_sync(FULL, incl, 31);
      rem -= min(rem, tot);
      if (rem == 0) break;
    }
  } else {
    // out-node: (e_out, e_in) with residual f_b; (e_out, u) uncapacitated
    const int e = x - nh - m;
    const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
    const int fb = N.f_b[e], ein = nh + e;
    const unsigned items = 1 + (end - beg);
    for (unsigned i0 = 0; i0 < items; i0 += 32) {
      const unsigned i = i0 + lane;
      long long r = 0;
      int y = -1;
      unsigned p = 0;
      if (i == 0) {
        if (fb > 0 && Lr[ein] == dt) { r = fb; y = ein; }
      } else if (i < items) {
        p = beg + i - 1;
        int u = N.pin[p];
        if (Lr[u] == dt) { r = rem; y = u; }
      }
      const long long incl = warp_incl_scan(r);
      const long long take = min(max(rem - (incl - r), 0LL), r);
      bool ap = false;
      if (take > 0) {
        if (i == 0) N.f_b[e] = fb - (int)take;
        else N.f_out[p] += (int)take;
        ap = deliver(N, y, take, epoch, sink_acc);
        a.pushes++;
      }
      warp_append(ap, y, nextl, ncnt);
      a.net += (i < items);
      const long long tot = __shfl_sync(FULL, incl, 31);
      rem -= min(rem, tot);
      if (rem == 0) break;
    }
  }
  bool want = false;
  if (lane == 0) {
    N.excess[x] = rem;
    if (rem > 0) {
      N.needrl[x] = 1;
      want = atomicExch(&N.stamp[x], epoch) != epoch;
    }
  }
  warp_append(want, x, nextl, ncnt);
  a.nodes += (lane == 0);
}

// New label of x after the pushes of the round: min over residual arcs
// (capped network) of d(v) + 1, from the labels of the round (Section 2,
// "relabel").  NL when x has no residual arc.
__device__ int warp_relabel(const NetDev& N, const int32_t* Lr, int x, unsigned lane, Acc& a) {
  const int NL = N.NL, nh = N.n_nodes, m = N.m_nets;
  int best = NL;
  if (x < nh) {
    const unsigned beg = N.node_off[x], end = N.node_off[x + 1];
    for (unsigned j = beg + lane; j < end; j += 32) {
      int2 it = N.inc[j];
      int w = N.net_w[it.x];
      if (w > N.f_in[it.y]) best = min(best, Lr[nh + it.x] + 1);
      if (N.f_out[it.y] > 0) best = min(best, Lr[nh + m + it.x] + 1);
      a.hyper++;
    }
  } else if (x < nh + m) {
    const int e = x - nh;
    const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
    if (lane == 0 && N.net_w[e] > N.f_b[e]) best = Lr[nh + m + e] + 1;
    for (unsigned p = beg + lane; p < end; p += 32) {
      if (N.f_in[p] > 0) best = min(best, Lr[N.pin[p]] + 1);
      a.net++;
    }
  } else {
    const int e = x - nh - m;
    const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
    if (lane == 0 && N.f_b[e] > 0) best = Lr[nh + e] + 1;
    for (unsigned p = beg + lane; p < end; p += 32) {
      best = min(best, Lr[N.pin[p]] + 1);
      a.net++;
    }
  }
  best = warp_min(best);
  return min(best, NL);
}

// ---------------------------------------------------------------------------
__device__ void phase_a(const NetDev& N, EngineCtl* E, const Sched& s, unsigned gwarp,
                        unsigned nwarps, unsigned lane, Acc& a) {
  const int32_t* Lr = lab_cur(N, s.lp);
  int32_t* Ln = lab_cur(N, s.lp ^ 1);
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (unsigned i = tid; i < s.rcnt; i += nth) {   // labels relabeled last round
    int x = N.list[L_RELAB][i];
    Ln[x] = Lr[x];
  }
  long long sink_acc = 0;
  for (unsigned w = gwarp; w < s.fcnt; w += nwarps)
    discharge(N, E, N.list[L_FRONT][w], Lr, s.epoch, lane, sink_acc, a);
  sink_acc = warp_sum(sink_acc);
  if (lane == 0 && sink_acc) atomicAdd(&E->c.flow, (unsigned long long)sink_acc);
}

__device__ void phase_b(const NetDev& N, EngineCtl* E, const Sched& s, unsigned gwarp,
                        unsigned nwarps, unsigned lane, Acc& a) {
  const int32_t* Lr = lab_cur(N, s.lp);
  int32_t* Ln = lab_cur(N, s.lp ^ 1);
  for (unsigned base = gwarp * 32; base < s.ncnt; base += nwarps * 32) {
    const unsigned i = base + lane;
    int y = -1, lab = N.NL;
    long long ex = 0;
    bool need = false;
    if (i < s.ncnt) {
      y = N.list[L_NEXT][i];
      long long d = N.delta[y];
      ex = N.excess[y] + d;
      if (d) N.delta[y] = 0;
      N.excess[y] = ex;
      lab = Lr[y];
      need = N.needrl[y] != 0;
      if (need) N.needrl[y] = 0;
      a.nodes++;
    }
    unsigned mask = __ballot_sync(FULL, need);
    while (mask) {
      const int l = __ffs(mask) - 1;
      mask &= mask - 1;
      const int yy = __shfl_sync(FULL, y, l);
      const int nl = warp_relabel(N, Lr, yy, lane, a);
      if ((int)lane == l) {
        lab = nl;
        Ln[yy] = nl;
      }
    }
    warp_append(need, y, N.list[L_RELAB], &E->cnt[L_RELAB]);
    warp_append(y >= 0 && ex > 0 && lab < N.NL, y, N.list[L_FRONT], &E->cnt[L_FRONT]);
  }
}

// Global relabel, step 1: exact labels start from the sinks (Section 2,
// "global relabeling").
__device__ void gr_init(const NetDev& N, EngineCtl* E, unsigned lane, Acc& a) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (unsigned x0 = tid - lane; x0 < (unsigned)N.NL; x0 += nth) {
    const unsigned x = x0 + lane;
    bool snk = false;
    if (x < (unsigned)N.NL) {
      snk = (N.flags[x] & kSink) != 0;
      int l = snk ? 0 : N.NL;
      N.lab0[x] = l;
      N.lab1[x] = l;
      N.needrl[x] = 0;
      if (snk && x < (unsigned)N.n_nodes) a.w += N.node_w[x];
    }
    warp_append(snk, (int)x, N.list[L_BFS], &E->cnt[L_BFS]);
  }
}

__device__ __forceinline__ bool gr_claim(const NetDev& N, int x, int d1, bool& act, Acc& a) {
  act = false;
  if (x < 0) return false;
  if (N.lab0[x] != N.NL) return false;
  if (N.flags[x] & kSource) return false;
  if (atomicCAS(&N.lab0[x], N.NL, d1) != N.NL) return false;
  N.lab1[x] = d1;
  act = N.excess[x] > 0;
  if (x < N.n_nodes) a.w += N.node_w[x];
  return true;
}

// Global relabel, one level: reverse BFS over residual arcs of the capped
// network; newly reached excess nodes become the frontier.
__device__ void gr_level(const NetDev& N, EngineCtl* E, const Sched& s, unsigned gwarp,
                         unsigned nwarps, unsigned lane, Acc& a) {
  const int nh = N.n_nodes, m = N.m_nets, d1 = s.level + 1;
  int32_t* bl = N.list[L_BFS];
  unsigned* bc = &E->cnt[L_BFS];
  int32_t* fl = N.list[L_FRONT];
  unsigned* fc = &E->cnt[L_FRONT];
  for (unsigned w = s.bfs_begin + gwarp; w < s.bfs_end; w += nwarps) {
    const int y = bl[w];
    if (y < nh) {
      // into a hypernode: (e_out, u) always, (e_in, u) when f_in > 0
      const unsigned beg = N.node_off[y], end = N.node_off[y + 1];
      for (unsigned j0 = beg; j0 < end; j0 += 32) {
        const unsigned j = j0 + lane;
        int c1 = -1, c2 = -1;
        if (j < end) {
          int2 it = N.inc[j];
          c1 = nh + m + it.x;
          if (N.f_in[it.y] > 0) c2 = nh + it.x;
          a.hyper++;
        }
        bool act1, act2;
        bool k1 = gr_claim(N, c1, d1, act1, a);
        bool k2 = gr_claim(N, c2, d1, act2, a);
        warp_append(k1, c1, bl, bc);
        warp_append(k2, c2, bl, bc);
        warp_append(act1, c1, fl, fc);
        warp_append(act2, c2, fl, fc);
      }
    } else {
      const bool is_in = y < nh + m;
      const int e = is_in ? y - nh : y - nh - m;
      const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
      const int w = N.net_w[e], fb = N.f_b[e];
      const unsigned items = 1 + (end - beg);
      for (unsigned i0 = 0; i0 < items; i0 += 32) {
        const unsigned i = i0 + lane;
        int c = -1;
        if (i == 0) {
          // into e_in: (e_out, e_in) when f_b > 0; into e_out: bridge when w > f_b
          if (is_in) { if (fb > 0) c = nh + m + e; }
          else if (w > fb) c = nh + e;
        } else if (i < items) {
          const unsigned p = beg + i - 1;
          // into e_in: (u, e_in) when f_in < w (capped); into e_out: (u, e_out) when f_out > 0
          if (is_in ? (N.f_in[p] < w) : (N.f_out[p] > 0)) c = N.pin[p];
          a.net++;
        }
        bool act;
        bool k = gr_claim(N, c, d1, act, a);
        warp_append(k, c, bl, bc);
        warp_append(act, c, fl, fc);
      }
    }
  }
}

// Source-side cut, step 1: seeds are the sources and every non-sink node with
// positive excess (Section 8.4, "Source-Side Cut").
__device__ void sr_init(const NetDev& N, EngineCtl* E, const Sched& s, unsigned lane, Acc& a) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (unsigned x0 = tid - lane; x0 < (unsigned)N.NL; x0 += nth) {
    const unsigned x = x0 + lane;
    bool seed = false;
    if (x < (unsigned)N.NL) {
      uint8_t f = N.flags[x];
      seed = (f & kSource) || (!(f & kSink) && N.excess[x] > 0);
      N.insr[x] = seed ? 1 : 0;
      if (seed) {
        N.stamp[x] = s.epoch;
        if (x < (unsigned)N.n_nodes) a.w += N.node_w[x];
      }
    }
    warp_append(seed, (int)x, N.list[L_BFS], &E->cnt[L_BFS]);
  }
}

__device__ __forceinline__ bool sr_claim(const NetDev& N, int y, unsigned epoch, Acc& a) {
  if (y < 0) return false;
  if (N.insr[y]) return false;
  if (atomicExch(&N.stamp[y], epoch) == epoch) return false;
  N.insr[y] = 1;
  if (y < N.n_nodes) a.w += N.node_w[y];
  return true;
}

// Source-side cut, one level: forward residual arcs with (u, e_in) uncapped.
__device__ void sr_level(const NetDev& N, EngineCtl* E, const Sched& s, unsigned gwarp,
                         unsigned nwarps, unsigned lane, Acc& a) {
  const int nh = N.n_nodes, m = N.m_nets;
  int32_t* bl = N.list[L_BFS];
  unsigned* bc = &E->cnt[L_BFS];
  for (unsigned w = s.bfs_begin + gwarp; w < s.bfs_end; w += nwarps) {
    const int x = bl[w];
    if (x < nh) {
      // out of a hypernode: (u, e_in) always, (u, e_out) when f_out > 0
      const unsigned beg = N.node_off[x], end = N.node_off[x + 1];
      for (unsigned j0 = beg; j0 < end; j0 += 32) {
        const unsigned j = j0 + lane;
        int c1 = -1, c2 = -1;
        if (j < end) {
          int2 it = N.inc[j];
          c1 = nh + it.x;
          if (N.f_out[it.y] > 0) c2 = nh + m + it.x;
          a.hyper++;
        }
        bool k1 = sr_claim(N, c1, s.epoch, a);
        bool k2 = sr_claim(N, c2, s.epoch, a);
        warp_append(k1, c1, bl, bc);
        warp_append(k2, c2, bl, bc);
      }
    } else {
      const bool is_in = x < nh + m;
      const int e = is_in ? x - nh : x - nh - m;
      const unsigned beg = N.net_off[e], end = N.net_off[e + 1];
      const int w = N.net_w[e], fb = N.f_b[e];
      const unsigned items = 1 + (end - beg);
      for (unsigned i0 = 0; i0 < items; i0 += 32) {
        const unsigned i = i0 + lane;
        int c = -1;
        if (i == 0) {
          // out of e_in: bridge when f_b < w; out of e_out: (e_out, e_in) when f_b > 0
          if (is_in) { if (fb < w) c = nh + m + e; }
          else if (fb > 0) c = nh + e;
        } else if (i < items) {
          const unsigned p = beg + i - 1;
          // out of e_in: (e_in, u) when f_in > 0; out of e_out: (e_out, u) always
          if (!is_in || N.f_in[p] > 0) c = N.pin[p];
          a.net++;
        }
        bool k = sr_claim(N, c, s.epoch, a);
        warp_append(k, c, bl, bc);
      }
    }
  }
}

// Distance from the original cut (reading of Section 6 "Region Growing" and
// Section 7 "Piercing"): breadth-first search inside the region from the
// vertices at distance 1.  Level list i holds the vertices at distance i + 1.
__device__ void dist_init(const NetDev& N, EngineCtl* E, unsigned lane) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (unsigned u0 = tid - lane; u0 < (unsigned)N.n_nodes; u0 += nth) {
    const unsigned u = u0 + lane;
    const bool seed = u >= 2 && u < (unsigned)N.n_nodes && N.node_dist[u] == 1;
    warp_append(seed, (int)u, N.list[L_BFS], &E->cnt[L_BFS]);
  }
}

__device__ void dist_level(const NetDev& N, EngineCtl* E, const Sched& s, unsigned gwarp,
                           unsigned nwarps, unsigned lane) {
  const int d2 = s.level + 2;
  int32_t* bl = N.list[L_BFS];
  unsigned* bc = &E->cnt[L_BFS];
  for (unsigned w = s.bfs_begin + gwarp; w < s.bfs_end; w += nwarps) {
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
        warp_append(claim, v, bl, bc);
      }
    }
  }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kEngineThreads) engine_kernel(NetDev N, EngineCtl* E, Params P) {
  __shared__ Sched ss;
  __shared__ Acc acc_sh;
  if (threadIdx.x == 0) acc_sh = Acc{0, 0, 0, 0, 0};
  const unsigned lane = lane_id();
  const unsigned wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const unsigned gwarp = blockIdx.x * nwb + wib, nwarps = gridDim.x * nwb;
  Acc a{0, 0, 0, 0, 0};
  bool run = grid_step(E, N, P, &ss, false, &acc_sh, 0);
  while (run) {
    int target = 0;
    switch (ss.state) {
      case ST_ROUND_A: phase_a(N, E, ss, gwarp, nwarps, lane, a); break;
      case ST_ROUND_B: phase_b(N, E, ss, gwarp, nwarps, lane, a); break;
      case ST_GR_INIT: gr_init(N, E, lane, a); target = 2; break;
      case ST_GR_LEVEL: gr_level(N, E, ss, gwarp, nwarps, lane, a); target = 2; break;
      case ST_SR_INIT: sr_init(N, E, ss, lane, a); target = 1; break;
      case ST_SR_LEVEL: sr_level(N, E, ss, gwarp, nwarps, lane, a); target = 1; break;
      case ST_DIST_INIT: dist_init(N, E, lane); break;
      case ST_DIST_LEVEL: dist_level(N, E, ss, gwarp, nwarps, lane); break;
      default: break;
    }
    if (a.w) {
      atomicAdd((unsigned long long*)&acc_sh.w, (unsigned long long)a.w);
      a.w = 0;
    }
    run = grid_step(E, N, P, &ss, true, &acc_sh, target);
  }
  // statistics
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
  }
}

}  // namespace hfp
