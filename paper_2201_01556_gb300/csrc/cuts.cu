// FlowCutter steps around the engine (Section 7, Algorithm 2; Section 8.4):
// engine state set-up, saturation of new sources, marking S_r / T_r as
// terminals, piercing-node selection, and cut outputs.
#include "kernels.cuh"

namespace hfp {

constexpr unsigned FULLC = 0xffffffffu;

// Engine state before a cooperative launch.  SETUP_PREP only opens a fresh
// stamp epoch and empties the frontier so that k_saturate can fill it.
__device__ void zero_phase_counters(EngineCtl& X) {
  for (int l = 0; l < C_COUNT; l++)
    for (int k = 0; k < 3; k++) X.cnt3[l][k] = 0;
  for (int k = 0; k < 3; k++) {
    X.flow3[k] = 0;
    X.w3[k] = 0;
    X.key3[k] = 0;
    X.node3[k] = -1;
  }
  X.gr_act[0] = 0;
  X.gr_act[1] = 0;
}

__global__ void k_engine_setup(EngineCtl* E, int mode, int32_t arg) {
  EngineCtl& X = *E;
  X.bar_count = 0;
  X.c.err = kDevOk;
  X.c.err_where = 0;
  switch (mode) {
    case SETUP_GR:
      zero_phase_counters(X);
      X.s.grs++;
      X.s.state = ST_GR_INIT;
      X.s.after_gr_exit = 0;
      X.s.wT = 0;
      X.s.wT_set = 1;
      break;
    case SETUP_ROUND:
      zero_phase_counters(X);
      // fresh epoch: the frontier was stamped by k_saturate under the last one
      X.s.epoch++;
      X.s.state = ST_ROUND_A;
      X.s.fcnt = X.cnt[0];
      X.s.fcnth = X.cnt[1];
      X.cnt[0] = 0;
      X.cnt[1] = 0;
      X.s.rcnt = 0;
      X.s.flow_ref = X.c.flow;
      X.s.stall = 0;
      break;
    case SETUP_SR:
      zero_phase_counters(X);
      X.s.state = ST_SR_INIT;
      X.s.epoch++;
      X.s.wS = 0;
      X.s.wS_set = 1;
      break;
    case SETUP_PREP:
      X.s.epoch++;
      X.cnt[0] = 0;
      X.cnt[1] = 0;
      break;
    case SETUP_DIST:
      zero_phase_counters(X);
      X.s.state = ST_DIST_INIT;
      break;
    case SETUP_BATCH:
      zero_phase_counters(X);
      break;
    case SETUP_GR_ADD:
      // T_r grows by the nodes reaching one new sink; wT is kept
      zero_phase_counters(X);
      X.s.state = ST_GR_ADD;
      X.s.seed = arg;
      X.s.after_gr_exit = 0;
      X.s.wT_set = 1;
      break;
    case SETUP_SR_ADD:
      // S_r grows by the reach of one new source; wS is kept
      zero_phase_counters(X);
      X.s.state = ST_SR_ADD;
      X.s.epoch++;
      X.s.seed = arg;
      X.s.wS_set = 1;
      break;
  }
}

// frontier append outside the engine: light nodes from the front of the list,
// heavy ones from the back (the engine's split-list layout)
__device__ __forceinline__ void front_append(bool want, int y, bool heavy, const NetDev& N,
                                             EngineCtl* E) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const unsigned ml = __ballot_sync(FULLC, want && !heavy);
  const unsigned mh = __ballot_sync(FULLC, want && heavy);
  if (ml) {
    const int ld = __ffs(ml) - 1;
    unsigned pos = 0;
    if ((int)lane == ld) pos = atomicAdd(&E->cnt[0], (unsigned)__popc(ml));
    pos = __shfl_sync(FULLC, pos, ld);
    if (want && !heavy) N.list[L_FRONT][pos + __popc(ml & lt)] = y;
  }
  if (mh) {
    const int ld = __ffs(mh) - 1;
    unsigned pos = 0;
    if ((int)lane == ld) pos = atomicAdd(&E->cnt[1], (unsigned)__popc(mh));
    pos = __shfl_sync(FULLC, pos, ld);
    if (want && heavy) N.list[L_FRONT][N.NL - 1 - (pos + __popc(mh & lt))] = y;
  }
}

// Saturate every residual arc out of the given (new) source hypernodes:
// (u, e_in) up to w(e) (the capped capacity) and (u, e_out) down to zero flow
// (Section 2, "Push-Relabel": all source edges are saturated).  Targets that
// are sinks add to the flow value; others receive excess and join the
// frontier.  A block per node; pushes of one node touch distinct nets.
__global__ void k_saturate(const NetDev N, EngineCtl* E, const int32_t* nodes, int32_t count) {
  const int nh = N.n_nodes, m = N.m_nets;
  const unsigned lane = threadIdx.x & 31;
  for (int k = blockIdx.x; k < count; k += gridDim.x) {
    const int u = nodes[k];
    const unsigned beg = N.node_off[u], end = N.node_off[u + 1];
    const unsigned epoch = E->s.epoch;
    unsigned long long sink_acc = 0;
    for (unsigned j0 = beg + (threadIdx.x - lane); j0 < end; j0 += blockDim.x) {
      const unsigned j = j0 + lane;
      bool a1 = false, a2 = false, h1 = false, h2 = false;
      int y1 = -1, y2 = -1;
      if (j < end) {
        int2 it = N.inc[j];
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
          if (f1 & kSink) sink_acc += d1;
          else {
            atomicAdd((unsigned long long*)&N.excess[y1], (unsigned long long)d1);
            a1 = atomicExch(&N.stamp[y1], epoch) != epoch;
          }
        }
        if (d2 > 0 && !(f2 & kSource)) {
          N.f_out[p] = 0;
          if (f2 & kSink) sink_acc += d2;
          else {
            atomicAdd((unsigned long long*)&N.excess[y2], (unsigned long long)d2);
            a2 = atomicExch(&N.stamp[y2], epoch) != epoch;
          }
        }
      }
      front_append(a1, y1, h1, N, E);
      front_append(a2, y2, h2, N, E);
    }
    if (sink_acc) atomicAdd(&E->c.flow, sink_acc);
  }
}

// S <- S_r + extra: every node of S_r and every extra hypernode becomes a
// source with label NL; their excess is absorbed (Algorithm 2, line 8).
// S <- S_r + extra.  With one new source v, v is the only source with
// residual arcs leaving S (S_r is closed under residual arcs, sources never
// receive pushes and push only when saturated), so the next S_r searches
// expand v alone besides the excess nodes; with several, every source.
__global__ void k_mark_sources(const NetDev N, EngineCtl* E, const int32_t* extra,
                               int32_t count) {
  const int NL = N.NL;
  if (blockIdx.x == 0 && threadIdx.x == 0) E->s.sr_one = count == 1 ? extra[0] + 1 : 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < NL + count; x += gridDim.x * blockDim.x) {
    int y;
    if (x < NL) {
      if (!N.insr[x]) continue;
      y = x;
    } else {
      y = extra[x - NL];
    }
    N.flags[y] = (N.flags[y] & kHeavy) | kSource;
    N.lab0[y] = NL;
    N.lab1[y] = NL;
    N.excess[y] = 0;
  }
}

// T <- T_r + extra (Algorithm 2, line 10).  T_r is {x : label < NL} right
// after a final global relabel.  The excess of a node that turns into a sink
// is added to the flow value (Section 8.4, "Sink-Side Piercing").  With one
// new sink v, v is the only sink a non-sink can have a residual arc into (no
// residual arc entered T_r, and sinks never push), so the next global
// relabels expand v alone; with several, every sink.
__global__ void k_mark_sinks(const NetDev N, EngineCtl* E, const int32_t* extra, int32_t count) {
  const int NL = N.NL;
  if (blockIdx.x == 0 && threadIdx.x == 0) E->s.gr_one = count == 1 ? extra[0] + 1 : 0;
  unsigned long long acc = 0;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < NL + count; x += gridDim.x * blockDim.x) {
    int y;
    if (x < NL) {
      if (N.lab0[x] >= NL) continue;
      y = x;
    } else {
      y = extra[x - NL];
    }
    if (N.flags[y] & kSink) continue;
    long long ex = N.excess[y];
    if (ex > 0) acc += (unsigned long long)ex;
    N.excess[y] = 0;
    N.flags[y] = (N.flags[y] & kHeavy) | kSink;
  }
  if (acc) atomicAdd(&E->c.flow, acc);
}

// Piercing candidates (Section 7, "Piercing"): pins of nets whose in-node
// (growing S) or out-node (growing T) is reachable from the growing side,
// not reachable themselves, not terminals of the other side, and light
// enough to keep the growing side within L.  Key, larger wins:
//   bit 54 valid, bit 53 no augmenting path, bits 32..52 signed distance
//   + 2^20, bits 0..31 ~fmix32(gid ^ seed) (smaller hash wins).
__device__ __forceinline__ unsigned long long pierce_key(const NetDev& N, int h, int grow_s,
                                                         long long max_w, long long w_reach,
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

__global__ void k_pierce_scan(const NetDev N, EngineCtl* E, int grow_s, long long max_w,
                              long long w_reach, uint32_t seed, int find,
                              unsigned long long below) {
  const int nh = N.n_nodes, m = N.m_nets, NL = N.NL;
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned long long best = find ? E->c.best_key : 0;
  unsigned long long mx = 0;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    const int node = grow_s ? nh + e : nh + m + e;
    const bool reach = grow_s ? N.insr[node] != 0 : N.lab0[node] < NL;
    if (!reach) continue;
    for (unsigned p = N.net_off[e] + lane; p < N.net_off[e + 1]; p += 32) {
      const int h = N.pin[p];
      unsigned long long k = pierce_key(N, h, grow_s, max_w, w_reach, seed);
      if (below && k >= below) k = 0;   // the next candidate after an earlier pick
      if (find) {
        if (k != 0 && k == best) E->c.best_node = h;
      } else if (k > mx) {
        mx = k;
      }
    }
  }
  if (!find) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long t = __shfl_xor_sync(FULLC, mx, o);
      mx = t > mx ? t : mx;
    }
    if (lane == 0 && mx) atomicMax(&E->c.best_key, mx);
  }
}

__global__ void k_pierce_reset(EngineCtl* E) {
  E->c.best_key = 0;
  E->c.best_node = -1;
}

__global__ void k_region_side(const NetDev N, int use_t, int32_t n_region, uint8_t* out) {
  const int NL = N.NL;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_region; i += gridDim.x * blockDim.x) {
    const int x = 2 + i;
    out[i] = use_t ? (N.lab0[x] < NL ? 1 : 0) : (N.insr[x] ? 0 : 1);
  }
}

__global__ void k_lawler_sink_side(const NetDev N, uint8_t* out) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N.NL; x += gridDim.x * blockDim.x)
    out[x] = N.lab0[x] < N.NL ? 1 : 0;
}

__global__ void k_cut_net_flags(const NetDev N, unsigned* flags) {
  const int nh = N.n_nodes, m = N.m_nets;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    flags[e] = (N.insr[nh + e] && !N.insr[nh + m + e]) ? 1u : 0u;
}

__global__ void k_cut_net_compact(const NetDev N, const unsigned* flags, const unsigned* pos,
                                  const int32_t* net_gid, int32_t* out, int32_t cap) {
  const int nh = N.n_nodes, m = N.m_nets;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    if (N.insr[nh + e] && !N.insr[nh + m + e] && (int)pos[e] < cap) out[pos[e]] = net_gid[e];
}

__global__ void k_inc_slots(const NetDev N, int32_t* out) {
  for (long long j = blockIdx.x * blockDim.x + threadIdx.x; j < N.p_pins;
       j += (long long)gridDim.x * blockDim.x)
    out[j] = N.inc[j].y;
}

// ---------------------------------------------------------------------------
static inline unsigned nblk(long long work, unsigned per, unsigned cap) {
  long long b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

void launch_engine_setup(EngineCtl* E, int mode, cudaStream_t st, int32_t arg) {
  k_engine_setup<<<1, 1, 0, st>>>(E, mode, arg);
  count_launches(1);
}

void launch_saturate(const NetDev& N, EngineCtl* E, const int32_t* nodes, int32_t count,
                     cudaStream_t st) {
  if (count > 0) {
    k_saturate<<<nblk(count, 1, 1024), 256, 0, st>>>(N, E, nodes, count);
    count_launches(1);
  }
}

void launch_mark_sources(const NetDev& N, EngineCtl* E, const int32_t* extra, int32_t count,
                         int sms, cudaStream_t st) {
  k_mark_sources<<<nblk((long long)N.NL + count, 256, sms * 8), 256, 0, st>>>(N, E, extra,
                                                                              count);
  count_launches(1);
}

void launch_mark_sinks(const NetDev& N, EngineCtl* E, const int32_t* extra, int32_t count,
                       int sms, cudaStream_t st) {
  k_mark_sinks<<<nblk((long long)N.NL + count, 256, sms * 8), 256, 0, st>>>(N, E, extra, count);
  count_launches(1);
}

void launch_pierce_select(const NetDev& N, EngineCtl* E, int grow_s, long long max_w,
                          long long w_reach, uint32_t seed, int sms, cudaStream_t st,
                          unsigned long long below) {
  k_pierce_reset<<<1, 1, 0, st>>>(E);
  count_launches(1);
  unsigned b = nblk((long long)N.m_nets * 32, 256, sms * 16);
  k_pierce_scan<<<b, 256, 0, st>>>(N, E, grow_s, max_w, w_reach, seed, 0, below);
  count_launches(1);
  k_pierce_scan<<<b, 256, 0, st>>>(N, E, grow_s, max_w, w_reach, seed, 1, below);
  count_launches(1);
}

void launch_region_side(const NetDev& N, int use_t, int32_t n_region, uint8_t* out, int sms,
                        cudaStream_t st) {
  if (n_region > 0) {
    k_region_side<<<nblk(n_region, 256, sms * 8), 256, 0, st>>>(N, use_t, n_region, out);
    count_launches(1);
  }
}

void launch_lawler_sink_side(const NetDev& N, uint8_t* out, int sms, cudaStream_t st) {
  k_lawler_sink_side<<<nblk(N.NL, 256, sms * 8), 256, 0, st>>>(N, out);
  count_launches(1);
}

void launch_cut_net_flags(const NetDev& N, unsigned* flags, int sms, cudaStream_t st) {
  if (N.m_nets > 0) {
    k_cut_net_flags<<<nblk(N.m_nets, 256, sms * 8), 256, 0, st>>>(N, flags);
    count_launches(1);
  }
}

void launch_cut_net_compact(const NetDev& N, const unsigned* flags, const unsigned* pos,
                            const int32_t* net_gid, int32_t* out, int32_t cap, int sms,
                            cudaStream_t st) {
  if (N.m_nets > 0) {
    k_cut_net_compact<<<nblk(N.m_nets, 256, sms * 8), 256, 0, st>>>(N, flags, pos, net_gid, out,
                                                                     cap);
    count_launches(1);
  }
}

void launch_inc_slots(const NetDev& N, int32_t* out, int sms, cudaStream_t st) {
  if (N.p_pins > 0) {
    k_inc_slots<<<nblk(N.p_pins, 256, sms * 8), 256, 0, st>>>(N, out);
    count_launches(1);
  }
}

__global__ void k_add_i64(const long long* a, const long long* b, long long* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = a[i] + (b ? b[i] : 0);
}

void launch_add_i64(const long long* a, const long long* b, long long* out, long long n, int sms,
                    cudaStream_t st) {
  if (n <= 0) return;
  k_add_i64<<<sms * 4, 256, 0, st>>>(a, b, out, n);
  count_launches(1);
}

}  // namespace hfp
