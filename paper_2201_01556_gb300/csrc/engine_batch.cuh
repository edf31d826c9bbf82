// Batched FlowCutter (included by engine.cu, inside namespace hfp).
//
// One cooperative launch solves many flow problems, e.g. all block pairs of
// a k-way refinement round (Section 5, "Parallel Scheduling").  The grid is
// cut into groups of G consecutive CTAs.  A group takes the next job from a
// device work queue and runs the whole of Algorithm 2 (Section 7) on it: the
// initial maximum flow, then, until the cut is balanced, the source-side cut
// S_r, the balance test, the piercing-node selection and the incremental
// augmentation after piercing.  The flow phases are the engine's own (the
// same push-relabel rounds, global relabels and breadth-first searches, with
// "grid" read as "group"); the FlowCutter steps are extra engine states.
// Every CTA of the group derives the next state itself after each group
// barrier, exactly as in engine_kernel, so no host round trip is left.
//
// The decisions are the ones of hfp_flowcutter: balanced iff both sides are
// within L, the better of two balanced sides is the one with the smaller
// heavier side (ties: the source side), S grows iff c(S_r) <= c(T_r), and the
// piercing key is pierce_key below.  Results are therefore identical to the
// one-problem-per-launch path.

// Piercing candidates (Section 7, "Piercing"): pins of nets whose in-node
// (growing S) or out-node (growing T) is reachable from the growing side,
// not reachable themselves, not terminals of the other side, and light
// enough to keep the growing side within L.  Key, larger wins:
//   bit 54 valid, bit 53 no augmenting path, bits 32..52 signed distance
//   + 2^20, bits 0..31 ~fmix32(gid ^ seed) (smaller hash wins).
__device__ __forceinline__ unsigned long long batch_pierce_key(const NetDev& N, int h,
                                                               int grow_s, long long max_w,
                                                               long long w_reach,
                                                               uint32_t seed) {
  const int NL = N.NL;
  const bool in_r = grow_s ? N.insr[h] != 0 : N.lab0[h] < NL;
  if (in_r) return 0;
  const uint8_t f = N.flags[h];
  if (f & (grow_s ? kSink : kSource)) return 0;
  if (w_reach + N.node_w[h] > max_w) return 0;
  const bool no_path = grow_s ? N.lab0[h] >= NL : N.insr[h] == 0;
  const int d = N.node_dist[h] < 0 ? kDistFar : N.node_dist[h];
  const int sd = (N.node_orig[h] == (grow_s ? 0 : 1)) ? d : -d;
  const uint32_t hh = fmix32((uint32_t)N.node_gid[h] ^ seed);
  return (1ull << 54) | ((unsigned long long)no_path << 53) |
         ((unsigned long long)(sd + (1 << 20)) << 32) | (unsigned long long)(0xffffffffu - hh);
}

// The stall rule of the incremental flows after a piercing.
__device__ __forceinline__ void incremental_stall(Params& P) {
  if (P.stall_rounds_pierce) P.stall_rounds = P.stall_rounds_pierce;
  else P.stall_adapt = 1;
}

__device__ __forceinline__ bool is_fc_state(int st) {
  return st == ST_FC_SAT || st == ST_FC_SEL || st == ST_FC_FIND || st == ST_FC_MARK_S ||
         st == ST_FC_MARK_T;
}

// FlowCutter control of one job, replicated in every CTA of the group.
enum FcStage : int { FC_FLOW = 0, FC_SR = 1, FC_DIST = 2, FC_TADD = 3 };
struct FcState {
  int stage;          // what the engine is computing when it reaches ST_DONE
  int grow_s;
  int it;             // flows computed so far (the first one included)
  int np;             // nodes pierced
  int node;           // node being pierced (source hypernode 0 at the start)
  int initial;        // the saturation of s that opens the first flow
  int dist_ready;
  int status;         // outcome once the job is finished
  int result_side;
  int finished;
  int nopath;         // the chosen piercing node has no augmenting path
  int pending;        // unsaturated source left by a lazy piercing (-1: none)
  int sat_gr;         // ST_FC_SAT saturates the pending source before a relabel
  int gr_pending;     // labels not exact since a lazy sink piercing
  unsigned long long best;
  long long source_weight;
};

// ---------------------------------------------------------------------------
// phases of the FlowCutter states (group-wide)

// Saturate every residual arc out of the new source u (Algorithm 2 line 8
// after the piercing; Section 2 "Push-Relabel" for s): (u, e_in) up to w(e),
// (u, e_out) down to zero flow.  Non-sink targets get the excess and join the
// frontier (stamped with the current epoch); sink targets add to the flow.
__device__ void fc_saturate(const NetDev& N, const Sched& L, const Team& T, const Slot& S, int u,
                            unsigned lane) {
  const int nh = N.n_nodes, m = N.m_nets;
  const unsigned beg = N.node_off[u], end = N.node_off[u + 1];
  unsigned long long sink_acc = 0;
  for (unsigned j0 = beg + T.gwarp * 32; j0 < end; j0 += T.nwarps * 32) {
    const unsigned j = j0 + lane;
    bool a1 = false, a2 = false, h1 = false, h2 = false;
    int y1 = -1, y2 = -1;
    if (j < end) {
      const int2 it = N.inc[j];
      const int e = it.x, p = it.y;
      y1 = nh + e;
      y2 = nh + m + e;
      const int w = N.net_w[e];
      const int d1 = w - N.f_in[p];
      const int d2 = N.f_out[p];
      const uint8_t f1 = N.flags[y1], f2 = N.flags[y2];
      h1 = (f1 & kHeavy) != 0;
      h2 = (f2 & kHeavy) != 0;
      if (d1 > 0 && !(f1 & kSource)) {
        N.f_in[p] = w;
        if (f1 & kSink) {
          sink_acc += d1;
        } else {
          atomicAdd((unsigned long long*)&N.excess[y1], (unsigned long long)d1);
          a1 = atomicExch(&N.stamp[y1], L.epoch) != L.epoch;
        }
      }
      if (d2 > 0 && !(f2 & kSource)) {
        N.f_out[p] = 0;
        if (f2 & kSink) {
          sink_acc += d2;
        } else {
          atomicAdd((unsigned long long*)&N.excess[y2], (unsigned long long)d2);
          a2 = atomicExch(&N.stamp[y2], L.epoch) != L.epoch;
        }
      }
    }
    append_split(a1, y1, h1, N.list[L_FRONT], S.c[C_FRONT], S.c[C_FRONTH], 0, 0, N.NL);
    append_split(a2, y2, h2, N.list[L_FRONT], S.c[C_FRONT], S.c[C_FRONTH], 0, 0, N.NL);
  }
  if (sink_acc) atomicAdd(S.flow, sink_acc);
}

// The marking scans read the membership of four nodes per load (insr bytes
// as one word, labels as an int4; both arrays are 256-byte aligned) and
// kMarkUnroll such loads per thread and step, in flight together.
constexpr int kMarkUnroll = 4;

__device__ __forceinline__ void mark_source(const NetDev& N, int y) {
  N.flags[y] = (N.flags[y] & kHeavy) | kSource;
  N.lab0[y] = N.NL;
  N.lab1[y] = N.NL;
  N.excess[y] = 0;
}

// S <- S_r + {u}: sources get label NL and lose their excess.
__device__ void fc_mark_sources(const NetDev& N, const Team& T, int u) {
  const int NL = N.NL, n4 = NL >> 2;
  const uint32_t* in4 = reinterpret_cast<const uint32_t*>(N.insr);
  for (int base = (int)T.tid; base < n4; base += kMarkUnroll * (int)T.nth) {
    uint32_t v[kMarkUnroll];
#pragma unroll
    for (int j = 0; j < kMarkUnroll; j++) {
      const int i = base + j * (int)T.nth;
      v[j] = i < n4 ? in4[i] : 0u;
    }
#pragma unroll
    for (int j = 0; j < kMarkUnroll; j++) {
      if (!v[j]) continue;
      const int x0 = 4 * (base + j * (int)T.nth);
#pragma unroll
      for (int b = 0; b < 4; b++)
        if ((v[j] >> (8 * b)) & 0xffu) mark_source(N, x0 + b);
    }
  }
  for (int x = 4 * n4 + (int)T.tid; x < NL; x += (int)T.nth)
    if (N.insr[x]) mark_source(N, x);
  if (T.tid == 0) mark_source(N, u);
}

__device__ __forceinline__ unsigned long long mark_sink(const NetDev& N, int y) {
  const uint8_t f = N.flags[y];
  if (f & kSink) return 0;
  const long long ex = N.excess[y];
  N.excess[y] = 0;
  N.flags[y] = (f & kHeavy) | kSink;
  return ex > 0 ? (unsigned long long)ex : 0ull;
}

// T <- T_r + {u} (T_r = {label < NL} after the final global relabel; u is
// outside it); the excess of a node that becomes a sink joins the flow
// (Section 8.4, "Sink-Side Piercing").
__device__ void fc_mark_sinks(const NetDev& N, const Team& T, const Slot& S, int u) {
  const int NL = N.NL, n4 = NL >> 2;
  const int4* l4 = reinterpret_cast<const int4*>(N.lab0);
  unsigned long long acc = 0;
  for (int base = (int)T.tid; base < n4; base += kMarkUnroll * (int)T.nth) {
    int4 v[kMarkUnroll];
#pragma unroll
    for (int j = 0; j < kMarkUnroll; j++) {
      const int i = base + j * (int)T.nth;
      v[j] = i < n4 ? l4[i] : make_int4(NL, NL, NL, NL);
    }
#pragma unroll
    for (int j = 0; j < kMarkUnroll; j++) {
      const int x0 = 4 * (base + j * (int)T.nth);
      if (v[j].x < NL) acc += mark_sink(N, x0);
      if (v[j].y < NL) acc += mark_sink(N, x0 + 1);
      if (v[j].z < NL) acc += mark_sink(N, x0 + 2);
      if (v[j].w < NL) acc += mark_sink(N, x0 + 3);
    }
  }
  for (int x = 4 * n4 + (int)T.tid; x < NL; x += (int)T.nth)
    if (N.lab0[x] < NL) acc += mark_sink(N, x);
  if (T.tid == 0) acc += mark_sink(N, u);
  if (acc) atomicAdd(S.flow, acc);
}

// Largest piercing key over the candidates and the node holding it, as the
// CTA's entry (sel_key, sel_node)[blockIdx.x] of the launch's BatchCtl (the
// group reduces its entries after the barrier; keys of distinct candidates
// differ in the hash bits, so the maximum has one holder).  A warp takes 32
// consecutive nets, one per lane, and walks the concatenated pin lists of the
// reachable ones 64 pins per step (two per lane, loads issued together), so
// a step costs one chain of dependent loads for up to 64 pins of 32 nets.  A reachable net whose pins all lie in the
// growing side's reachable set gets its net_done flag: the marking that
// follows this selection makes all of them terminals, so the net never has
// a candidate again and later scans skip it.  Every thread of the CTA must
// call it.
constexpr unsigned kSelBig = 256;   // pins above which the CTA walks a net
constexpr int kSelBigCap = 256;     // CTA queue of such nets (more: walked by warps)

__device__ void fc_pierce_select(const NetDev& N, const Team& T, BatchCtl* B, const FcJob& J,
                                 const FcState& F, long long w_reach, unsigned lane,
                                 unsigned* walked) {
  __shared__ unsigned long long sk[32];
  __shared__ int sn[32];
  __shared__ int qbuf[kEngineThreads / 32][64];   // per warp: reachable nets not yet walked
  __shared__ int bigq[kSelBigCap];                  // per CTA: reachable nets of many pins
  __shared__ unsigned bign;
  __shared__ unsigned bincl[32];
  __shared__ int bout[32];
  const int nh = N.n_nodes, m = N.m_nets, NL = N.NL;
  if (threadIdx.x == 0) bign = 0;
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  int* qb = qbuf[threadIdx.x >> 5];
  unsigned long long best = 0;
  int bnode = -1;
  // Pins of the nets e (one per lane, -1: none), 32 pins per step.
  auto walk = [&](int e) {
    const unsigned nw = __popc(__ballot_sync(FULL, e >= 0));
    if (lane == 0) atomicAdd(walked, nw);
    unsigned beg = 0, sz = 0;
    if (e >= 0) {
      beg = N.net_off[e];
      sz = N.net_off[e + 1] - beg;
    }
    unsigned incl = sz;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(FULL, incl, o);
      if ((int)lane >= o) incl += t;
    }
    const unsigned total = __shfl_sync(FULL, incl, 31);
    const unsigned excl = incl - sz;
    bool outside = false;   // this lane's net has a pin outside the reachable set
    // pin q of the walk: its slot (0xffffffff: none)
    auto slot_of = [&](unsigned q) {
      int own = 0;   // owner = number of lanes whose inclusive end is <= q
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const unsigned v = __shfl_sync(FULL, incl, own + step - 1);
        if (v <= q) own += step;
      }
      own = own < 31 ? own : 31;
      const unsigned ob = __shfl_sync(FULL, beg, own), oe = __shfl_sync(FULL, excl, own);
      return q < total ? ob + (q - oe) : 0xffffffffu;
    };
    // whether this lane's net has pins among lanes [lo, hi) of window q0
    auto mine = [&](unsigned q0, unsigned ballot) {
      if (!sz || excl >= q0 + 32 || incl <= q0) return false;
      const unsigned lo = excl > q0 ? excl - q0 : 0u;
      const unsigned hi = incl - q0 < 32u ? incl - q0 : 32u;
      const unsigned mask = (hi == 32u ? FULL : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
      return (ballot & mask) != 0;
    };
    for (unsigned q0 = 0; q0 < total; q0 += 64) {
      const unsigned pa = slot_of(q0 + lane), pb = slot_of(q0 + 32 + lane);
      const int ha = pa != 0xffffffffu ? N.pin[pa] : -1;
      const int hb = pb != 0xffffffffu ? N.pin[pb] : -1;
      bool oa = false, ob2 = false;
      if (ha >= 0) oa = F.grow_s ? N.insr[ha] == 0 : N.lab0[ha] >= NL;
      if (hb >= 0) ob2 = F.grow_s ? N.insr[hb] == 0 : N.lab0[hb] >= NL;
      if (oa) {
        const unsigned long long k = batch_pierce_key(N, ha, F.grow_s, J.max_w, w_reach, J.seed);
        if (k > best) {
          best = k;
          bnode = ha;
        }
      }
      if (ob2) {
        const unsigned long long k = batch_pierce_key(N, hb, F.grow_s, J.max_w, w_reach, J.seed);
        if (k > best) {
          best = k;
          bnode = hb;
        }
      }
      const unsigned ba = __ballot_sync(FULL, oa), bb = __ballot_sync(FULL, ob2);
      if (mine(q0, ba) || mine(q0 + 32, bb)) outside = true;
    }
    if (sz && !outside && N.net_done) N.net_done[e] = 1;
  };
  // The reach of 4 batches of 32 nets is loaded at once; the reachable nets
  // not yet done are queued per warp and walked 32 at a time, so the walks
  // run with full warps however the reachable nets spread over the ids.
  // Nets of more than kSelBig pins go to the CTA's queue instead (a warp
  // would walk a net of thousands of pins alone while the group waits).
  constexpr int kBatches = 4;
  unsigned qn = 0;
  for (unsigned e00 = T.gwarp * 32 * kBatches; e00 < (unsigned)m;
       e00 += T.nwarps * 32 * kBatches) {
    bool rch[kBatches];
#pragma unroll
    for (int j = 0; j < kBatches; j++) {
      const unsigned e = e00 + j * 32 + lane;
      rch[j] = false;
      if (e < (unsigned)m) {
        const int node = F.grow_s ? nh + (int)e : nh + m + (int)e;
        const bool done = N.net_done && N.net_done[e];
        const bool reach = F.grow_s ? N.insr[node] != 0 : N.lab0[node] < NL;
        rch[j] = reach && !done;
      }
    }
#pragma unroll 1
    for (int j = 0; j < kBatches; j++) {
      if (!__ballot_sync(FULL, rch[j])) continue;
      const unsigned e = e00 + j * 32 + lane;
      if (rch[j] && N.net_off[e + 1] - N.net_off[e] > kSelBig) {
        const unsigned slot = atomicAdd(&bign, 1u);
        if (slot < (unsigned)kSelBigCap) {
          bigq[slot] = (int)e;
          rch[j] = false;
        }
      }
      const unsigned msk = __ballot_sync(FULL, rch[j]);
      if (rch[j]) qb[qn + __popc(msk & lt)] = (int)e;
      qn += __popc(msk);
      __syncwarp();
      if (qn >= 32) {
        const int e = qb[lane];
        const int rest = lane + 32 < qn ? qb[lane + 32] : -1;
        __syncwarp();
        if (lane + 32 < qn) qb[lane] = rest;
        qn -= 32;
        __syncwarp();
        walk(e);
      }
    }
  }
  if (qn) walk(lane < qn ? qb[lane] : -1);
  // the CTA's nets of many pins, up to 32 per step: the CTA walks their
  // concatenated pin lists blockDim.x pins at a time
  __syncthreads();
  const unsigned nbig = min(bign, (unsigned)kSelBigCap);
  for (unsigned b0 = 0; b0 < nbig; b0 += 32) {
    if (threadIdx.x < 32) {
      const unsigned t = threadIdx.x;
      unsigned sz = 0;
      if (b0 + t < nbig) {
        const int e = bigq[b0 + t];
        sz = N.net_off[e + 1] - N.net_off[e];
      }
      unsigned incl = sz;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned v = __shfl_up_sync(FULL, incl, o);
        if ((int)t >= o) incl += v;
      }
      bincl[t] = incl;
      bout[t] = 0;
    }
    __syncthreads();
    const unsigned total = bincl[31];
    for (unsigned q0 = 0; q0 < total; q0 += blockDim.x) {
      const unsigned q = q0 + threadIdx.x;
      if (q < total) {
        int own = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (bincl[own + step - 1] <= q) own += step;
        own = own < 31 ? own : 31;
        const int e = bigq[b0 + own];
        const unsigned first = own ? bincl[own - 1] : 0u;
        const int h = N.pin[N.net_off[e] + (q - first)];
        const bool out = F.grow_s ? N.insr[h] == 0 : N.lab0[h] >= NL;
        if (out) {
          bout[own] = 1;
          const unsigned long long k = batch_pierce_key(N, h, F.grow_s, J.max_w, w_reach, J.seed);
          if (k > best) {
            best = k;
            bnode = h;
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x < 32 && b0 + threadIdx.x < nbig && !bout[threadIdx.x] && N.net_done)
      N.net_done[bigq[b0 + threadIdx.x]] = 1;
    __syncthreads();   // bincl and bout are rewritten by the next step
  }
  if (threadIdx.x == 0 && nbig) atomicAdd(walked, nbig);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long tk = __shfl_xor_sync(FULL, best, o);
    const int tn = __shfl_xor_sync(FULL, bnode, o);
    if (tk > best) {
      best = tk;
      bnode = tn;
    }
  }
  const unsigned w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    sk[w] = best;
    sn[w] = bnode;
  }
  __syncthreads();
  if (w == 0) {
    best = lane < nw ? sk[lane] : 0ull;
    bnode = lane < nw ? sn[lane] : -1;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long tk = __shfl_xor_sync(FULL, best, o);
      const int tn = __shfl_xor_sync(FULL, bnode, o);
      if (tk > best) {
        best = tk;
        bnode = tn;
      }
    }
    if (lane == 0) {
      B->sel_key[blockIdx.x] = best;
      B->sel_node[blockIdx.x] = bnode;
    }
  }
}

// The group's largest key and its node from the entries of its G CTAs
// (first CTA of the group: c0).  Warp 0 of the calling CTA; the result is
// in lane 0.
__device__ void fc_select_reduce(const BatchCtl* B, unsigned c0, int G, unsigned lane,
                                 unsigned long long& key, int& node) {
  unsigned long long best = 0;
  int bnode = -1;
  for (int r = (int)lane; r < G; r += 32) {
    const unsigned long long k = __ldcg(&B->sel_key[c0 + r]);
    const int h = __ldcg(&B->sel_node[c0 + r]);
    if (k > best) {
      best = k;
      bnode = h;
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long tk = __shfl_xor_sync(FULL, best, o);
    const int tn = __shfl_xor_sync(FULL, bnode, o);
    if (tk > best) {
      best = tk;
      bnode = tn;
    }
  }
  key = best;
  node = bnode;
}

// ---------------------------------------------------------------------------
// control (thread 0 of every CTA of the group, on identical inputs)

__device__ void fc_finish(Sched& L, FcState& F, int status) {
  F.status = status;
  F.finished = 1;
  L.state = ST_DONE;
}

// The engine reached ST_DONE: continue Algorithm 2.
__device__ void fc_on_done(Sched& L, FcState& F, const FcJob& J, const Ctl* c) {
  const int err = ld_volatile_int(&c->err);
  if (err != kDevOk) {
    fc_finish(L, F, 100 + err);
    return;
  }
  switch (F.stage) {
    case FC_FLOW:
      // source-side cut of the new flow (SETUP_SR)
      F.stage = FC_SR;
      L.state = ST_SR_INIT;
      L.epoch++;
      L.wS = 0;
      L.wS_set = 1;
      return;
    case FC_DIST:
      F.dist_ready = 1;
      L.state = ST_FC_SEL;
      return;
    default:
      break;   // FC_SR, FC_TADD: S_r and T_r are current
  }
  // FC_SR: S_r and T_r of the current flow are known (Algorithm 2, lines 3-6)
  const long long W = J.total_w, Lm = J.max_w;
  const long long wS = L.wS, wT = L.wT;
  if (J.flow_bound >= 0 && (long long)L.flow > J.flow_bound) {
    fc_finish(L, F, -6 /* HFP_ABORTED_WORSE */);
    return;
  }
  const bool balS = wS <= Lm && W - wS <= Lm;
  const bool balT = wT <= Lm && W - wT <= Lm;
  if (balS || balT) {
    bool use_t;
    if (balS && balT) {
      const long long mS = wS > W - wS ? wS : W - wS;
      const long long mT = wT > W - wT ? wT : W - wT;
      use_t = mT < mS;
    } else {
      use_t = !balS;
    }
    F.result_side = use_t ? 1 : 0;
    F.source_weight = use_t ? W - wT : wS;
    fc_finish(L, F, 0);
    return;
  }
  if (F.it >= J.max_it) {
    fc_finish(L, F, -4 /* HFP_ERR_ITER_LIMIT */);
    return;
  }
  F.grow_s = wS <= wT ? 1 : 0;
  if (!F.dist_ready) {
    F.stage = FC_DIST;     // SETUP_DIST
    L.state = ST_DIST_INIT;
  } else {
    L.state = ST_FC_SEL;
  }
}

// After a FlowCutter phase and its barrier.
//
// Terminal boundaries.  After S <- S_r + {v}, the only source with a residual
// arc to a non-source is v: S_r was closed under residual arcs, no push ever
// enters a source (its label is N_L and no label exceeds N_L), and a source
// pushes only when it is saturated, which is v's own step.  Symmetrically,
// after T <- T_r + {v} only v can have a residual arc from a non-sink: no
// residual arc entered T_r from outside, and sinks never push, so no arc into
// T gains residual capacity later.  So the global relabels seed the last
// pierced sink alone (every sink still gets label 0) and the S_r searches the
// last pierced source alone plus the excess nodes (every source still joins
// S_r): the same labels and cuts as seeding every terminal, without
// expanding the interiors of S and T, which grow to half the network.
__device__ void fc_advance(Sched& L, FcState& F, const Snap& q, const FcJob& J, Params& P,
                           bool recorder) {
  switch (L.state) {
    case ST_FC_SAT:
      L.flow += q.flow;
      F.stage = FC_FLOW;
      if (!F.initial) incremental_stall(P);
      if (F.initial || F.sat_gr) {
        // first flow, or a sink piercing after a lazy one: the labels are
        // built by a global relabel (SETUP_GR)
        F.initial = 0;
        F.sat_gr = 0;
        begin_gr(L);
        L.after_gr_exit = 0;
      } else if (F.gr_pending || P.pierce_relabel) {
        // labels are stale after a lazy sink piercing, or the tuning asks for
        // exact labels before the rounds: relabel first
        F.gr_pending = 0;
        begin_gr(L);
        L.after_gr_exit = 0;
        F.it++;
      } else {
        // the new excess is the frontier; labels stay valid (SETUP_ROUND)
        L.epoch++;
        L.state = round_state(P);
        L.fsel = L_FRONT;
        L.fcnt = q.c[C_FRONT];
        L.fcnth = q.c[C_FRONTH];
        L.rcnt = 0;
        L.flow_ref = L.flow;
        L.stall = 0;
        F.it++;
      }
      break;
    case ST_FC_SEL:
      // q.key / q.node: the group's largest key and its holder
      if (q.key == 0) {
        fc_finish(L, F, -5 /* HFP_NO_BALANCED_CUT */);
        break;
      }
      F.best = q.key;
      F.node = q.node;
      F.nopath = (int)((F.best >> 53) & 1ull);
      if (recorder && F.np < J.pierce_cap) {
        if (J.pierce_node) J.pierce_node[F.np] = q.node;
        if (J.pierce_side) J.pierce_side[F.np] = (int8_t)(F.grow_s ? 0 : 1);
      }
      F.np++;
      L.state = F.grow_s ? ST_FC_MARK_S : ST_FC_MARK_T;
      break;
    case ST_FC_MARK_S:
      L.epoch++;           // SETUP_PREP / SETUP_SR_ADD: fresh stamps
      L.sr_one = F.node + 1;   // the one source with residual arcs out of S
      if (F.nopath) {
        // lazy piercing (hfp_flowcutter's rule): the preflow stays maximum,
        // S_r grows by the node's reach, its arcs wait for a sink piercing
        F.pending = F.node;
        F.stage = FC_SR;
        F.it++;
        L.state = ST_SR_ADD;
        L.seed = F.node;
        L.wS_set = 1;
      } else {
        F.pending = -1;
        L.state = ST_FC_SAT;
      }
      break;
    case ST_FC_MARK_T:
      L.flow += q.flow;    // excess absorbed by the new sinks
      L.gr_one = F.node + 1;   // the one sink with residual arcs into T
      F.stage = FC_FLOW;
      F.it++;
      incremental_stall(P);   // the flows from here on are incremental
      if (F.nopath) {
        // lazy piercing: the flow and S_r stay, T_r grows by a reverse search
        // from the node; the next flow computation relabels first
        F.stage = FC_TADD;
        F.gr_pending = 1;
        L.state = ST_GR_ADD;
        L.seed = F.node;
        L.after_gr_exit = 0;
        L.wT_set = 1;
        break;
      }
      F.gr_pending = 0;
      if (F.pending >= 0) {
        // the unsaturated source may now reach T: saturate it first
        F.node = F.pending;
        F.pending = -1;
        F.sat_gr = 1;
        L.epoch++;
        L.state = ST_FC_SAT;
      } else {
        begin_gr(L);       // SETUP_GR: labels are no longer lower bounds
        L.after_gr_exit = 0;
      }
      break;
    default:
      L.state = ST_DONE;
  }
}

// Count-up barrier of a group on BatchCtl (job hand-out), bounded like
// grid_barrier; false on expiry (B->err set).
__device__ bool group_sync(BatchCtl* B, int gid, unsigned target,
                           unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    red_release_add(&B->gbar[gid], 1u);
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (!count_reached(ld_acquire(&B->gbar[gid]), target)) {
      if ((++spins & 255u) == 0) {
        if (ld_volatile_int(&B->err) != 0) { ok = 0; break; }
        const unsigned long long t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > timeout_ns) {
          atomicCAS(&B->err, 0, 1);
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

// Barrier of a group that is one thread-block cluster: the counter is a
// word in the shared memory of the cluster's first CTA (`ctr`, a
// shared::cluster address), arrivals are cluster-scope release reductions
// and the wait is a cluster-scope acquire spin, so the group's global-memory
// writes before the barrier are visible to the whole group after it.  The
// wait is bounded like grid_barrier: every 256 spins it polls *err (raised by
// another CTA) and globaltimer; on expiry *err = code (and *where = 1 when
// given) and false is returned.
__device__ bool cluster_barrier(unsigned ctr, unsigned target, int* err, int code, int* where,
                                unsigned long long timeout_ns) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    dsmem_red_release_add(ctr, 1u);
    unsigned spins = 0;
    unsigned long long t0 = 0;
    while (!count_reached(dsmem_ld_acquire(ctr), target)) {
      if ((++spins & 255u) == 0) {
        if (ld_volatile_int(err) != 0) { ok = 0; break; }
        const unsigned long long t = globaltimer();
        if (t0 == 0) t0 = t;
        else if (t - t0 > timeout_ns) {
          atomicCAS(err, 0, code);
          if (where) *where = 1;
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

// The barrier a group uses: the cluster-resident counter when the group is a
// cluster (ctr != kNoCluster, running sequence *cseq over the launch), else
// the job's global counter (sequence *bar_seq within the job).
constexpr unsigned kNoCluster = 0xffffffffu;

__device__ __forceinline__ bool job_barrier(EngineCtl* E, unsigned ctr, unsigned& cseq,
                                            unsigned& bar_seq, unsigned G,
                                            unsigned long long timeout_ns) {
  if (ctr != kNoCluster)
    return cluster_barrier(ctr, G * ++cseq, &E->c.err, kDevTimeout, &E->c.err_where, timeout_ns);
  return grid_barrier(E, G * ++bar_seq, timeout_ns);
}

__device__ void run_phase_batch(const NetDev& N, EngineCtl* E, BatchCtl* B, const Sched& L,
                                const FcState& F, const FcJob& J, const Team& T, unsigned lane,
                                Acc& a, long long* w_sh, const Params& P) {
  const Slot S = slot_of(E, L.phase);
  switch (L.state) {
    case ST_FC_SAT: fc_saturate(N, L, T, S, F.node, lane); break;
    case ST_FC_SEL:
      fc_pierce_select(N, T, B, J, F, F.grow_s ? L.wS : L.wT, lane, S.c[C_RELAB]);
      break;
    case ST_FC_MARK_S: fc_mark_sources(N, T, F.node); break;
    case ST_FC_MARK_T: fc_mark_sinks(N, T, S, F.node); break;
    default: run_phase(N, E, L, T, lane, a, w_sh, P); break;
  }
}

// Group time per state of the running job, kept by thread 0 of its first CTA.
struct BatchClock {
  unsigned long long t;
  unsigned long long ns[kStateSlots];
  unsigned cnt[kStateSlots];
  unsigned long long lin[kStateSlots], hin[kStateSlots];   // light / heavy input nodes
};

// Input of a phase of state st: the frontier (rounds), the next list (apply
// and relabel) or the breadth-first-search level (light, heavy).
__device__ __forceinline__ void phase_input(const Sched& L, int st, unsigned long long& li,
                                            unsigned long long& hi) {
  if (st == ST_ROUND_A || st == ST_ROUND || st == ST_FLUSH) {
    li = L.fcnt;
    hi = L.fcnth;
  } else if (st == ST_ROUND_B) {
    li = L.ncnt;
    hi = L.ncnth;
  } else if (st == ST_GR_LEVEL || st == ST_SR_LEVEL || st == ST_DIST_LEVEL) {
    li = L.bfs_end - L.bfs_begin;
    hi = L.bfsh_end - L.bfsh_begin;
  } else {
    li = hi = 0;
  }
}

// `walked`: nets whose pins a selection phase walked (counted as its light
// input).
__device__ __forceinline__ void batch_tick(BatchClock& bc, int st, const Sched& L,
                                           unsigned walked) {
  const unsigned long long t = globaltimer();
  unsigned long long li, hi;
  phase_input(L, st, li, hi);
  if (st == ST_FC_SEL) li = walked;
  st = st < kStateSlots ? st : kStateSlots - 1;
  bc.ns[st] += t - bc.t;
  bc.cnt[st]++;
  bc.lin[st] += li;
  bc.hin[st] += hi;
  bc.t = t;
}

// One job by one group of G CTAs (rank = position in the group).
__device__ void fc_run_job(FcJob* job, const Params& P0, int rank, int G, unsigned lane,
                           Sched& L, FcState& F, NetDev& N, Params& P, long long* w_sh,
                           Clock& ck, SoloSh& solo, unsigned ctr, unsigned& cseq,
                           BatchClock& bc, BatchCtl* B) {
  const unsigned wib = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const Team T{rank * nwb + wib, G * nwb, rank * blockDim.x + threadIdx.x, G * blockDim.x,
               (unsigned)rank, (unsigned)G};
  EngineCtl* E = job->E;
  unsigned long long t_start = 0;
  if (threadIdx.x == 0) {
    t_start = globaltimer();
    N = job->N;
    P = P0;
    P.gr_work = job->gr_work;
    if (!N.delta1) P.fused_rounds = 0;   // buffers of this network
    if (!N.gq) P.async_gr = 0;
    if (rank == 0) {
      for (int k = 0; k < kStateSlots; k++) {
        bc.ns[k] = 0;
        bc.cnt[k] = 0;
        bc.lin[k] = 0;
        bc.hin[k] = 0;
      }
      bc.t = t_start;
    }
    load_sched(L, E);
    L.flow = *(const volatile unsigned long long*)&E->c.flow;
    F = FcState{FC_FLOW, 0, 1, 0, 0, 1, job->dist_ready, 0, 0, 0, 0, -1, 0, 0, 0ull, 0ll};
    // SETUP_PREP, then the saturation of s opens the first flow
    L.epoch++;
    L.state = ST_FC_SAT;
    L.sr_one = 1;   // S = {s}, T = {t}
    L.gr_one = 2;
    *w_sh = 0;
  }
  __syncthreads();
  Acc a{0, 0, 0, 0, 0};
  unsigned bar_seq = 0;
  const bool lead = rank == 0;
  for (;;) {
    const int st = L.state;
    if (st == ST_DONE) break;
    if (solo_next(L, P)) {
      if (lead) {
        solo_phases(N, E, P, L, lane, a, w_sh, ck, solo);
        if (threadIdx.x == 0) store_sched(E, L);
      }
      const bool ok = job_barrier(E, ctr, cseq, bar_seq, G, P.timeout_ns);
      if (threadIdx.x == 0) {
        if (lead) batch_tick(bc, ST_TAIL, L, 0);
        if (!lead) load_sched(L, E);
        if (!ok) L.state = ST_DONE;
        if (L.state == ST_DONE && !F.finished) fc_on_done(L, F, *job, &E->c);
      }
      __syncthreads();
      continue;
    }
    if (lead && threadIdx.x == 0)
      clear_slot(E, (L.phase + 1) % 3, st == ST_GR_INIT || st == ST_GR_ADD);
    run_phase_batch(N, E, B, L, F, *job, T, lane, a, w_sh, P);
    __syncthreads();
    if (threadIdx.x == 0) flush_weight(E, L.phase, w_sh);
    const bool ok = job_barrier(E, ctr, cseq, bar_seq, G, P.timeout_ns);
    unsigned long long sel_key = 0;
    int sel_node = -1;
    if (st == ST_FC_SEL && threadIdx.x < 32)
      fc_select_reduce(B, blockIdx.x - (unsigned)rank, G, lane, sel_key, sel_node);
    if (threadIdx.x == 0) {
      if (!ok) {
        if (lead) batch_tick(bc, st, L, 0);
        L.state = ST_DONE;
        fc_on_done(L, F, *job, &E->c);
      } else {
        Snap q = take_snap(E, L.phase);
        if (lead) batch_tick(bc, st, L, st == ST_FC_SEL ? q.c[C_RELAB] : 0u);
        if (st == ST_FC_SEL) {
          q.key = sel_key;
          q.node = sel_node;
        }
        if (is_fc_state(st)) fc_advance(L, F, q, *job, P, lead);
        else advance(L, q, P, N, &E->c);
        L.phase++;
        if (L.state == ST_DONE && !F.finished) fc_on_done(L, F, *job, &E->c);
      }
    }
    __syncthreads();
  }
  // statistics and results (the group leader)
  if (a.hyper) atomicAdd(&E->c.items_hyper, a.hyper);
  if (a.net) atomicAdd(&E->c.items_net, a.net);
  if (a.nodes) atomicAdd(&E->c.node_visits, a.nodes);
  if (a.pushes) atomicAdd(&E->c.pushes, a.pushes);
  if (lead && threadIdx.x == 0) {
    // later calls on the network seed every terminal again
    L.gr_one = 0;
    L.sr_one = 0;
    store_sched(E, L);
    E->c.flow = L.flow;
    E->c.rounds = L.rounds;
    E->c.global_relabels = L.grs;
    E->c.gr_levels = L.gr_levels;
    if (L.wS_set) E->c.wS = L.wS;
    if (L.wT_set) E->c.wT = L.wT;
    job->status = F.status;
    job->iterations = F.it;
    job->n_pierced = F.np;
    job->result_side = F.result_side;
    job->flow = (long long)L.flow;
    job->source_weight = F.source_weight;
    job->device_ns = globaltimer() - t_start;
    job->group_ctas = G;
    for (int k = 0; k < kStateSlots; k++) {
      job->st_ns[k] = bc.ns[k];
      job->st_cnt[k] = bc.cnt[k];
      job->st_lin[k] = bc.lin[k];
      job->st_hin[k] = bc.hin[k];
    }
  }
}

// The batched launch.  The grid is cut into groups: the first `big` groups
// of Gb CTAs, then groups of G CTAs.  The host sorts the jobs largest first;
// group g starts on job g (so the big groups take the largest problems) and
// every group then takes the next job from the queue until none is left.
// With `cluster` set (uniform groups only) the launch has clusters of G CTAs
// and each group is one cluster (group barriers in distributed shared
// memory); otherwise it is a cooperative launch and groups synchronise
// through global counters.
__global__ void __launch_bounds__(kEngineThreads, 2) fc_batch_kernel(FcJob* jobs, int n_jobs,
                                                                  BatchCtl* B, int G, int Gb,
                                                                  int big, int n_groups,
                                                                  Params P0, int cluster) {
  __shared__ Sched L;
  __shared__ FcState F;
  __shared__ NetDev N;
  __shared__ Params P;
  __shared__ long long w_sh;
  __shared__ Clock ck;
  __shared__ SoloSh solo;
  __shared__ unsigned job_sh;
  __shared__ unsigned gbar_sh;   // the group's barrier counter (cluster rank 0's is used)
  __shared__ BatchClock bclk;
  const int big_ctas = big * Gb;
  int gid, rank, Gg;
  if ((int)blockIdx.x < big_ctas) {
    gid = blockIdx.x / Gb;
    rank = blockIdx.x % Gb;
    Gg = Gb;
  } else {
    const int x = blockIdx.x - big_ctas;
    gid = big + x / G;
    rank = x % G;
    Gg = G;
  }
  const unsigned lane = lane_id();
  unsigned ctr = kNoCluster;
  if (threadIdx.x == 0) {
    ck.t_last = globaltimer();
    gbar_sh = 0;
  }
  if (cluster) {
    cluster_sync_all();           // every counter is zero before the first arrival
    ctr = dsmem_addr(&gbar_sh, 0);
  }
  unsigned gseq = 0, cseq = 0;
  unsigned j = (unsigned)gid;
  for (;;) {
    if (j >= (unsigned)n_jobs) break;
    fc_run_job(&jobs[j], P0, rank, Gg, lane, L, F, N, P, &w_sh, ck, solo, ctr, cseq, bclk, B);
    // hand-out of the next job (the queue starts after the first job of every group)
    if (rank == 0 && threadIdx.x == 0) B->gjob[gid] = n_groups + atomicAdd(&B->next, 1u);
    const bool ok = cluster ? cluster_barrier(ctr, Gg * ++cseq, &B->err, 1, nullptr, P0.timeout_ns)
                            : group_sync(B, gid, Gg * ++gseq, P0.timeout_ns);
    if (!ok) break;
    if (threadIdx.x == 0) job_sh = *(const volatile unsigned*)&B->gjob[gid];
    __syncthreads();
    j = job_sh;
  }
  // no CTA of a cluster exits while another may still read its shared memory
  if (cluster) cluster_sync_all();
}

// A bounded wait that nothing completes: the barrier `which` (0: the engine's
// grid barrier, 1: a batched group's barrier in global memory, 2: a cluster
// barrier in the first CTA's shared memory; the launch is then one cluster)
// waits for one arrival more than the launch has CTAs, so only its timeout
// ends it.  Every CTA leaves with the error word set and nothing in flight.
__global__ void wait_selftest_kernel(EngineCtl* E, BatchCtl* B, int which,
                                     unsigned long long timeout_ns) {
  __shared__ unsigned ctr_sh;
  const unsigned target = gridDim.x + 1;
  if (which == 2) {
    if (threadIdx.x == 0) ctr_sh = 0;
    cluster_sync_all();
    cluster_barrier(dsmem_addr(&ctr_sh, 0), target, &B->err, 1, nullptr, timeout_ns);
    cluster_sync_all();   // no CTA leaves while another may read its shared memory
  } else if (which == 1) {
    group_sync(B, 0, target, timeout_ns);
  } else {
    grid_barrier(E, target, timeout_ns);
  }
}
