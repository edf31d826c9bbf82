// k-way flow-based refinement (Section 4, Algorithm 1; Section 5; Section 6):
// a device-resident hypergraph with its vertex -> nets incidence, region
// growing for a block pair, refine_block_pair (region, flow network,
// FlowCutter, moves) and a synchronous refinement round with the
// apply-moves rules of Section 5.
//
// Readings (shared with the oracle): the region of pair (i, j) is grown
// inside each block by breadth-first search from the block's pins of the
// pair's cut nets (distance 1) up to distance delta, taking vertices level by
// level in ascending id order while the block's share stays within
//   max(0, floor((100 + alpha_eps_pct) * ceil((c(Vi)+c(Vj))/2) / 100) - c(Vj));
// the first vertex that does not fit ends that block's growth.  A round
// refines every pair against the same partition, then applies the move sets
// with Delta_exp >= 0 in descending Delta_exp (ties: ascending (i, j)),
// dropping stale moves, skipping a set that would push a growing block past
// the bound, and reverting a set whose actual gain is negative.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace hfp;

namespace hfp {

namespace {

inline unsigned nb(long long work, unsigned per, unsigned cap) {
  long long b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// incidence of H
__global__ void k_vdeg(int32_t m, const uint32_t* net_off, const int32_t* pins, unsigned* deg) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < (long long)net_off[m];
       j += (long long)gridDim.x * blockDim.x)
    atomicAdd(&deg[pins[j]], 1u);
}

__global__ void k_vfill(int32_t m, const uint32_t* net_off, const int32_t* pins,
                        const unsigned* off, unsigned* cursor, int32_t* vnet) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw)
    for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) {
      const int v = pins[j];
      vnet[off[v] + atomicAdd(&cursor[v], 1u)] = (int32_t)e;
    }
}

// warp per vertex: sort its net ids (rank sort; ids are distinct)
__global__ void k_vsort(int32_t n, const unsigned* off, int32_t* vnet, int32_t* tmp) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned v = gw; v < (unsigned)n; v += nw) {
    const unsigned beg = off[v], d = off[v + 1] - beg;
    if (d <= 1) continue;
    if (d <= 32) {
      const int mine = lane < d ? vnet[beg + lane] : 0x7fffffff;
      unsigned rank = 0;
      for (unsigned k = 0; k < d; k++) rank += (__shfl_sync(0xffffffffu, mine, k) < mine);
      __syncwarp();
      if (lane < d) vnet[beg + rank] = mine;
    } else {
      for (unsigned i = lane; i < d; i += 32) {
        const int mine = vnet[beg + i];
        unsigned rank = 0;
        for (unsigned k = 0; k < d; k++) rank += (vnet[beg + k] < mine);
        tmp[beg + rank] = mine;
      }
      __syncwarp();
      for (unsigned i = lane; i < d; i += 32) vnet[beg + i] = tmp[beg + i];
    }
  }
}

__global__ void k_unit_weights(int32_t n, int32_t* w) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) w[v] = 1;
}

// ---------------------------------------------------------------------------
// pair region

// candidates in ascending order with exclusive weight prefix wpre: the first
// ones whose inclusive prefix fits in the budget are taken
__global__ void k_take(unsigned cnt, const int32_t* cand, const unsigned* wpre,
                       const int32_t* node_w, long long budget, uint8_t* in_b,
                       unsigned* taken) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int v = cand[i];
    if ((long long)wpre[i] + node_w[v] <= budget) {
      in_b[v] = 1;
      atomicAdd(taken, 1u);
    }
  }
}

// next BFS level inside the block: from taken vertices of level d, pins of
// their nets on the same side still unlabelled get level d + 1
__global__ void k_next_level(unsigned cnt, const int32_t* cand, const uint32_t* vnet_off,
                             const int32_t* vnet, const uint32_t* net_off, const int32_t* pins,
                             const int32_t* side, int s, int32_t* lev, int d1) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < cnt; i += nw) {
    const int v = cand[i];
    for (unsigned t = vnet_off[v]; t < vnet_off[v + 1]; t++) {
      const int e = vnet[t];
      for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) {
        const int u = pins[j];
        if (side[u] == s && lev[u] == 0) atomicCAS(&lev[u], 0, d1);
      }
    }
  }
}

__global__ void k_region_dist(unsigned cnt, const int32_t* region, const int32_t* lev,
                              int32_t* dist) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    dist[i] = lev[region[i]];
}

// original cut of the pair on the network's nets (s counts as side 0, t as 1)
__global__ void k_pair_cut(const NetDev N, unsigned long long* cut) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0;
  for (unsigned e = gw; e < (unsigned)N.m_nets; e += nw) {
    bool a = false, b = false;
    for (unsigned p0 = N.net_off[e]; p0 < N.net_off[e + 1]; p0 += 32) {
      const unsigned p = p0 + lane;
      int s = -1;
      if (p < N.net_off[e + 1]) {
        const int h = N.pin[p];
        s = h == 0 ? 0 : (h == 1 ? 1 : N.node_orig[h]);
      }
      a |= __any_sync(0xffffffffu, s == 0);
      b |= __any_sync(0xffffffffu, s == 1);
    }
    if (lane == 0 && a && b) acc += (unsigned long long)N.net_w[e];
  }
  if (acc) atomicAdd(cut, acc);
}

// moves of a pair: region vertices whose final side differs from the
// original one, in region order: (vertex, from block, to block)
// region vertex i moves when its final side differs from its block (bi: 0)
__global__ void k_move_flags(unsigned cnt, const int32_t* region, const int32_t* part, int32_t bi,
                             const uint8_t* fin, unsigned* flag) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    flag[i] = (int)fin[i] != (part[region[i]] == bi ? 0 : 1) ? 1u : 0u;
}

__global__ void k_move_fill(unsigned cnt, const int32_t* region, const uint8_t* fin,
                            const unsigned* flag, const unsigned* pos, int32_t bi, int32_t bj,
                            int32_t* moves) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    if (flag[i]) {
      const unsigned q = pos[i];
      moves[3 * q] = region[i];
      moves[3 * q + 1] = fin[i] ? bi : bj;
      moves[3 * q + 2] = fin[i] ? bj : bi;
    }
}

// ---------------------------------------------------------------------------
// block lists: the vertices and the nets of every block, ascending, so that
// the preparation of a pair works on its two blocks only

// block mask of every net (k <= 64), a warp per net
__global__ void k_net_mask(int32_t m, const uint32_t* net_off, const int32_t* pins,
                           const int32_t* part, unsigned long long* mask) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    unsigned long long mk = 0;
    for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) mk |= 1ull << part[pins[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mk |= __shfl_xor_sync(0xffffffffu, mk, o);
    if (lane == 0) mask[e] = mk;
  }
}

// Stable grouping of items by block (counting sort in tiles of kGrpTile
// items, one CTA each): item i belongs to every block of its mask (a vertex:
// its block; a net: the blocks of its pins).  k_grp_count writes the count
// of block b in tile t to C[b * T + t]; after an exclusive scan of C (block
// major), k_grp_place puts item i of block b at C[b * T + t] + the number of
// earlier items of its tile in b, so every block's list is ascending.
constexpr int kGrpTile = 512;

__device__ __forceinline__ unsigned long long grp_mask(int32_t i, int32_t n, const int32_t* part,
                                                       const unsigned long long* nmask) {
  if (i >= n) return 0ull;
  return part ? 1ull << part[i] : nmask[i];
}

__global__ void __launch_bounds__(kGrpTile) k_grp_count(int32_t n, const int32_t* part,
                                                        const unsigned long long* nmask, int k,
                                                        unsigned T, unsigned* C) {
  __shared__ unsigned cnt[64];
  if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long mk = grp_mask(blockIdx.x * kGrpTile + threadIdx.x, n, part, nmask);
  while (mk) {
    atomicAdd(&cnt[__ffsll(mk) - 1], 1u);
    mk &= mk - 1;
  }
  __syncthreads();
  if ((int)threadIdx.x < k) C[threadIdx.x * T + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void __launch_bounds__(kGrpTile) k_grp_place(int32_t n, const int32_t* part,
                                                        const unsigned long long* nmask, int k,
                                                        unsigned T, const unsigned* C,
                                                        int32_t* out) {
  __shared__ unsigned wc[kGrpTile / 32][64];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5, lt = (1u << lane) - 1u;
  const int32_t i = blockIdx.x * kGrpTile + threadIdx.x;
  const unsigned long long mk = grp_mask(i, n, part, nmask);
  for (int b = 0; b < k; b++) {
    const unsigned bal = __ballot_sync(0xffffffffu, (mk >> b) & 1ull);
    if (lane == 0) wc[w][b] = __popc(bal);
  }
  __syncthreads();
  if ((int)threadIdx.x < k) {
    unsigned run = 0;
    for (int q = 0; q < kGrpTile / 32; q++) {
      const unsigned v = wc[q][threadIdx.x];
      wc[q][threadIdx.x] = run;
      run += v;
    }
  }
  __syncthreads();
  for (int b = 0; b < k; b++) {
    const bool in = (mk >> b) & 1ull;
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    if (in) out[C[b * T + blockIdx.x] + wc[w][b] + __popc(bal & lt)] = i;
  }
}

// side of the vertices of one block (s = 0 / 1) or back to -1 with level 0
// and not taken (s < 0)
__global__ void k_list_side(unsigned cnt, const int32_t* list, int s, int32_t* side, int32_t* lev,
                            uint8_t* in_b) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int v = list[i];
    side[v] = s;
    if (s < 0) {
      lev[v] = 0;
      in_b[v] = 0;
    }
  }
}

// level 1 from the nets of block bi that also hold pins of block bj (the
// pair's cut nets): their pins of either block, a warp per net
__global__ void k_level1_list(unsigned cnt, const int32_t* nets, const unsigned long long* mask,
                              int32_t bi, int32_t bj, const uint32_t* net_off, const int32_t* pins,
                              const int32_t* side, int32_t* lev) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned i = gw; i < cnt; i += nw) {
    const int e = nets[i];
    if (!((mask[e] >> bj) & 1ull)) continue;
    for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) {
      const int v = pins[j];
      if (side[v] >= 0) lev[v] = 1;
    }
  }
  (void)bi;
}

// flag[i] = the vertex list[i] has level d (d >= 0) / is taken (d < 0)
__global__ void k_list_flag(unsigned cnt, const int32_t* list, const int32_t* lev,
                            const uint8_t* in_b, int d, unsigned* flag) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    const int v = list[i];
    flag[i] = d >= 0 ? (lev[v] == d ? 1u : 0u) : (unsigned)in_b[v];
  }
}

// flag[i] = net nets[i] has no pin in block b
__global__ void k_net_not_in(unsigned cnt, const int32_t* nets, const unsigned long long* mask,
                             int32_t b, unsigned* flag) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    flag[i] = ((mask[nets[i]] >> b) & 1ull) ? 0u : 1u;
}

__global__ void k_list_scatter(unsigned cnt, const int32_t* list, const unsigned* flag,
                               const unsigned* pos, int32_t* out, const int32_t* node_w,
                               unsigned* wout) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x)
    if (flag[i]) {
      out[pos[i]] = list[i];
      if (wout) wout[pos[i]] = (unsigned)node_w[list[i]];
    }
}

// pins of a net in each block of its mask, at cnt[noff[e] + rank of the block
// in the mask] (a warp per net)
__global__ void k_mask_popc(int32_t m, const unsigned long long* mask, unsigned* out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x)
    out[e] = __popcll(mask[e]);
}

__global__ void k_net_block_counts(int32_t m, const uint32_t* net_off, const int32_t* pins,
                                   const int32_t* part, const unsigned long long* mask,
                                   const unsigned* noff, unsigned* cnt) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    const unsigned long long mk = mask[e];
    for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) {
      const int b = part[pins[j]];
      atomicAdd(&cnt[noff[e] + __popcll(mk & ((1ull << b) - 1ull))], 1u);
    }
  }
}

// block list offsets from the scanned tile counts: out[b] = start of block b,
// out[k] = total
__global__ void k_grp_offsets(const unsigned* C, unsigned T, int k, const unsigned* total,
                              unsigned* out) {
  if ((int)threadIdx.x < k) out[threadIdx.x] = C[threadIdx.x * T];
  if (threadIdx.x == 0) out[k] = *total;
}

// merge of two disjoint ascending lists into one ascending list
__global__ void k_merge_sorted(const int32_t* a, unsigned na, const int32_t* b, unsigned nb,
                               int32_t* out) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < na + nb;
       i += gridDim.x * blockDim.x) {
    const bool in_a = i < na;
    const int32_t v = in_a ? a[i] : b[i - na];
    const int32_t* o = in_a ? b : a;
    unsigned lo = 0, hi = in_a ? nb : na;   // elements of the other list below v
    while (lo < hi) {
      const unsigned mid = (lo + hi) >> 1;
      if (o[mid] < v) lo = mid + 1;
      else hi = mid;
    }
    out[(in_a ? i : i - na) + lo] = v;
  }
}

// ---------------------------------------------------------------------------
// round: connectivity, quotient graph, apply moves (k <= 64: block masks)
__global__ void k_connectivity(int32_t m, const uint32_t* net_off, const int32_t* pins,
                               const int32_t* net_w, const int32_t* part,
                               unsigned long long* out, unsigned long long* pair_nets,
                               unsigned long long* pair_w, int32_t k) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long acc = 0;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    unsigned long long mask = 0;
    for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) mask |= 1ull << part[pins[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    const int lam = __popcll(mask);
    if (lane == 0 && lam > 1) acc += (unsigned long long)(lam - 1) * net_w[e];
    if (pair_nets && lam > 1) {
      // pairs of blocks present, lane-strided over the first block
      for (int a = lane; a < k; a += 32) {
        if (!((mask >> a) & 1ull)) continue;
        unsigned long long rest = mask >> (a + 1);
        while (rest) {
          const int b = a + 1 + __ffsll(rest) - 1;
          rest &= rest - 1;
          atomicAdd(&pair_nets[a * k + b], 1ull);
          atomicAdd(&pair_w[a * k + b], (unsigned long long)net_w[e]);
        }
      }
    }
  }
  if (lane == 0 && acc) atomicAdd(out, acc);
}

// stale check and weight change of a move set
__global__ void k_apply_check(unsigned cnt, const int32_t* mv, const int32_t* part,
                              const int32_t* node_w, uint8_t* valid, long long* dw,
                              unsigned* nvalid, int32_t* moved_to, unsigned epoch,
                              unsigned* moved_stamp) {
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x) {
    const int v = mv[3 * q], a = mv[3 * q + 1], b = mv[3 * q + 2];
    const bool ok = part[v] == a;
    valid[q] = ok;
    if (ok) {
      atomicAdd((unsigned long long*)&dw[a], (unsigned long long)(-(long long)node_w[v]));
      atomicAdd((unsigned long long*)&dw[b], (unsigned long long)node_w[v]);
      atomicAdd(nvalid, 1u);
      moved_to[v] = b;
      moved_stamp[v] = epoch;
    }
  }
}

// actual gain (Section 5, "Apply Moves"): per net touched by a valid move,
// w(e) times the number of the two blocks it leaves minus the number it
// newly reaches.  Each net is claimed once through its stamp.
__global__ void k_apply_gain(unsigned cnt, const int32_t* mv, const uint8_t* valid,
                             const uint32_t* vnet_off, const int32_t* vnet,
                             const uint32_t* net_off, const int32_t* pins, const int32_t* net_w,
                             const int32_t* part, const int32_t* moved_to,
                             const unsigned* moved_stamp, unsigned* net_stamp, unsigned epoch,
                             int32_t bi, int32_t bj, long long* gain) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  long long acc = 0;
  for (unsigned q = gw; q < cnt; q += nw) {
    if (!valid[q]) continue;
    const int v = mv[3 * q];
    for (unsigned t = vnet_off[v]; t < vnet_off[v + 1]; t++) {
      const int e = vnet[t];
      int claim = 0;
      if (lane == 0) claim = atomicExch(&net_stamp[e], epoch) != epoch;
      claim = __shfl_sync(0xffffffffu, claim, 0);
      if (!claim) continue;
      int ca0 = 0, cb0 = 0, ca1 = 0, cb1 = 0;
      for (unsigned j = net_off[e] + lane; j < net_off[e + 1]; j += 32) {
        const int u = pins[j];
        const int before = part[u];
        const int after = moved_stamp[u] == epoch ? moved_to[u] : before;
        ca0 += before == bi;
        cb0 += before == bj;
        ca1 += after == bi;
        cb1 += after == bj;
      }
      ca0 = __reduce_add_sync(0xffffffffu, ca0);
      cb0 = __reduce_add_sync(0xffffffffu, cb0);
      ca1 = __reduce_add_sync(0xffffffffu, ca1);
      cb1 = __reduce_add_sync(0xffffffffu, cb1);
      if (lane == 0)
        acc += (long long)net_w[e] * ((ca0 > 0) + (cb0 > 0) - (ca1 > 0) - (cb1 > 0));
    }
  }
  if (lane == 0 && acc) atomicAdd((unsigned long long*)gain, (unsigned long long)acc);
}

__global__ void k_apply_commit(unsigned cnt, const int32_t* mv, const uint8_t* valid,
                               int32_t* part) {
  for (unsigned q = blockIdx.x * blockDim.x + threadIdx.x; q < cnt; q += gridDim.x * blockDim.x)
    if (valid[q]) part[mv[3 * q]] = mv[3 * q + 2];
}

__global__ void k_block_weights(int32_t n, const int32_t* part, const int32_t* node_w,
                                unsigned long long* bw) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd(&bw[part[v]], (unsigned long long)node_w[v]);
}

}  // namespace

}  // namespace hfp

namespace {

hfp_status hg_set_device(hfp_hgraph* hg) {
  CK(cudaSetDevice(hg->ctx->device));
  return HFP_OK;
}

}  // namespace

HFP_API hfp_status hfp_hgraph_create(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                                     hfp_hgraph** out) {
  if (!out) return fail(HFP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx || !H || H->n < 0 || H->m < 0 || !H->net_off || (H->m > 0 && (!H->pins || !H->net_w)))
    return fail(HFP_ERR_INVALID, "bad hypergraph");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  const int32_t n = H->n, m = H->m;
  uint32_t P = 0;
  if (mem == HFP_MEM_HOST) {
    P = H->net_off[m];
  } else {
    uint32_t* h = (uint32_t*)ctx->pinned_small;
    CK(cudaMemcpyAsync(h, H->net_off + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    P = h[0];
  }
  if (P >= (1u << 31)) return fail(HFP_ERR_INVALID, "too many pins");
  hfp_hgraph* hg = new hfp_hgraph();
  hg->ctx = ctx;
  hg->n = n;
  hg->m = m;
  hg->p = P;
  const size_t sz[] = {align_up(sizeof(uint32_t) * (m + 1)), align_up(sizeof(int32_t) * P),
                       align_up(sizeof(int32_t) * (m > 0 ? m : 1)),
                       align_up(sizeof(int32_t) * (n > 0 ? n : 1)),
                       align_up(sizeof(uint32_t) * (n + 1)), align_up(sizeof(int32_t) * P)};
  size_t total = 0;
  for (size_t b : sz) total += b;
  if (cudaMallocAsync(&hg->arena, total, st) != cudaSuccess) {
    delete hg;
    return fail(HFP_ERR_OOM, "cannot allocate the hypergraph");
  }
  char* q = (char*)hg->arena;
  hg->net_off = (uint32_t*)q; q += sz[0];
  hg->pins = (int32_t*)q; q += sz[1];
  hg->net_w = (int32_t*)q; q += sz[2];
  hg->node_w = (int32_t*)q; q += sz[3];
  hg->vnet_off = (uint32_t*)q; q += sz[4];
  hg->vnet = (int32_t*)q;
  const cudaMemcpyKind kind = mem == HFP_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(hg->net_off, H->net_off, sizeof(uint32_t) * (m + 1), kind, st));
  if (P) CK(cudaMemcpyAsync(hg->pins, H->pins, sizeof(int32_t) * P, kind, st));
  if (m) CK(cudaMemcpyAsync(hg->net_w, H->net_w, sizeof(int32_t) * m, kind, st));
  if (H->node_w) {
    if (n) CK(cudaMemcpyAsync(hg->node_w, H->node_w, sizeof(int32_t) * n, kind, st));
  } else if (n) {
    k_unit_weights<<<nb(n, 256, ctx->sms * 8), 256, 0, st>>>(n, hg->node_w);
    count_launches(1);
  }
  // vertex -> nets incidence, ascending net ids
  {
    DevBuf cursor, tmp, scr, tot;
    CK(cursor.alloc(sizeof(unsigned) * (n > 0 ? n : 1), st));
    CK(tmp.alloc(sizeof(int32_t) * (P > 0 ? P : 1), st));
    CK(scr.alloc(sizeof(unsigned) * (scan_scratch_words(n + 1) + 8), st));
    CK(tot.alloc(sizeof(unsigned), st));
    CK(cudaMemsetAsync(hg->vnet_off, 0, sizeof(unsigned) * (n + 1), st));
    if (P) {
      k_vdeg<<<nb(P, 256, ctx->sms * 8), 256, 0, st>>>(m, hg->net_off, hg->pins, hg->vnet_off);
      count_launches(1);
    }
    scan_exclusive(hg->vnet_off, n + 1, scr.as<unsigned>(), tot.as<unsigned>(), st);
    CK(cudaMemsetAsync(cursor.p, 0, sizeof(unsigned) * (n > 0 ? n : 1), st));
    if (m) {
      k_vfill<<<nb((long long)m * 32, 256, ctx->sms * 16), 256, 0, st>>>(
          m, hg->net_off, hg->pins, hg->vnet_off, cursor.as<unsigned>(), hg->vnet);
      count_launches(1);
    }
    if (n) {
      k_vsort<<<nb((long long)n * 32, 256, ctx->sms * 16), 256, 0, st>>>(n, hg->vnet_off, hg->vnet,
                                                                         tmp.as<int32_t>());
      count_launches(1);
    }
  }
  // total vertex weight
  {
    DevBuf bw;
    CK(bw.alloc(sizeof(unsigned long long), st));
    CK(cudaMemsetAsync(bw.p, 0, sizeof(unsigned long long), st));
    DevBuf zero;
    CK(zero.alloc(sizeof(int32_t) * (n > 0 ? n : 1), st));
    CK(cudaMemsetAsync(zero.p, 0, sizeof(int32_t) * (n > 0 ? n : 1), st));
    if (n) {
      k_block_weights<<<nb(n, 256, ctx->sms * 8), 256, 0, st>>>(n, zero.as<int32_t>(), hg->node_w,
                                                                bw.as<unsigned long long>());
      count_launches(1);
    }
    unsigned long long h = 0;
    CK(cudaMemcpyAsync(&h, bw.p, sizeof(h), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    hg->total_w = (int64_t)h;
  }
  ctx->refs.fetch_add(1);
  *out = hg;
  return HFP_OK;
}

HFP_API void hfp_hgraph_destroy(hfp_hgraph* hg) {
  if (!hg) return;
  hfp_ctx* c = hg->ctx;
  cudaSetDevice(c->device);
  for (hfp_ctx* h : hg->prep) hfp_ctx_destroy(h);
  if (hg->arena) cudaFreeAsync(hg->arena, c->stream);
  cudaStreamSynchronize(c->stream);
  delete hg;
  hfp_ctx_destroy(c);   // releases the reference taken at creation
}

namespace {

// One pair: region, network, FlowCutter, moves (device) and Delta_exp.
// moves_dev receives up to cap triples; res->n_moves is the count.
// Buffers of region growing, reused by the pairs of a round.  side, lev and
// in_b cover all vertices; a pair sets them for its two blocks and puts them
// back (-1, 0, 0) when its network is built.
struct RegionScratch {
  DevBuf side, lev, flag, pos, cand, wts, scr, tot, inb, taken, cut, rv, nets2, netlist, vlist;
  hfp_status alloc(hfp_hgraph* hg, cudaStream_t st) {
    const size_t n = hg->n > 0 ? hg->n : 1, m = hg->m > 0 ? hg->m : 1;
    const size_t nm = n > m ? n : m;
    CK(side.alloc(sizeof(int32_t) * n, st));
    CK(lev.alloc(sizeof(int32_t) * n, st));
    CK(flag.alloc(sizeof(unsigned) * nm, st));
    CK(pos.alloc(sizeof(unsigned) * nm, st));
    CK(cand.alloc(sizeof(int32_t) * n, st));
    CK(wts.alloc(sizeof(unsigned) * n, st));
    CK(scr.alloc(sizeof(unsigned) * (scan_scratch_words((unsigned)nm) + 8), st));
    CK(tot.alloc(sizeof(unsigned), st));
    CK(inb.alloc(n, st));
    CK(taken.alloc(sizeof(unsigned), st));
    CK(cut.alloc(sizeof(unsigned long long), st));
    CK(rv.alloc(sizeof(int32_t) * n, st));
    CK(nets2.alloc(sizeof(int32_t) * m, st));
    CK(netlist.alloc(sizeof(int32_t) * m, st));
    CK(vlist.alloc(sizeof(int32_t) * n, st));
    CK(cudaMemsetAsync(side.p, 0xFF, sizeof(int32_t) * n, st));
    CK(cudaMemsetAsync(lev.p, 0, sizeof(int32_t) * n, st));
    CK(cudaMemsetAsync(inb.p, 0, n, st));
    return HFP_OK;
  }
};

// The vertices and the nets of every block in ascending order, the nets'
// block masks and the block weights, for one partition (k <= 64).
struct BlockLists {
  DevBuf nmask, C, bv, bn, offs, noff, cnt;
  std::vector<unsigned> bv_off, bn_off;     // k + 1 each
  std::vector<unsigned long long> bw;       // k
  bool counts = false;                      // noff / cnt built
  // pins of every (net, block) pair, for the second construction algorithm
  hfp_status build_counts(hfp_hgraph* hg, const int32_t* part) {
    if (counts) return HFP_OK;
    cudaStream_t st = hg->ctx->stream;
    const int m = hg->m, sms = hg->ctx->sms;
    CK(noff.alloc(sizeof(unsigned) * (m + 1), st));
    unsigned total = 0;
    if (m) {
      DevBuf scr, tot;
      CK(scr.alloc(sizeof(unsigned) * (scan_scratch_words((unsigned)m) + 8), st));
      CK(tot.alloc(sizeof(unsigned), st));
      k_mask_popc<<<nb(m, 256, sms * 8), 256, 0, st>>>(m, nmask.as<unsigned long long>(),
                                                       noff.as<unsigned>());
      count_launches(1);
      scan_exclusive(noff.as<unsigned>(), (unsigned)m, scr.as<unsigned>(), tot.as<unsigned>(), st);
      CK(cudaMemcpyAsync(&total, tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    CK(cnt.alloc(sizeof(unsigned) * (total > 0 ? total : 1), st));
    CK(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned) * (total > 0 ? total : 1), st));
    if (m) {
      k_net_block_counts<<<nb((long long)m * 32, 256, sms * 16), 256, 0, st>>>(
          m, hg->net_off, hg->pins, part, nmask.as<unsigned long long>(), noff.as<unsigned>(),
          cnt.as<unsigned>());
      count_launches(1);
    }
    counts = true;
    return HFP_OK;
  }
  hfp_status build(hfp_hgraph* hg, const int32_t* part, int32_t k) {
    hfp_ctx* ctx = hg->ctx;
    cudaStream_t st = ctx->stream;
    const int n = hg->n, m = hg->m, sms = ctx->sms;
    const unsigned Tv = (unsigned)((n + kGrpTile - 1) / kGrpTile);
    const unsigned Tn = (unsigned)((m + kGrpTile - 1) / kGrpTile);
    const size_t cmax = (size_t)k * (Tv > Tn ? Tv : Tn) + 1;
    DevBuf scr, tot, dbw;
    CK(nmask.alloc(sizeof(unsigned long long) * (m > 0 ? m : 1), st));
    CK(C.alloc(sizeof(unsigned) * cmax, st));
    CK(bv.alloc(sizeof(int32_t) * (n > 0 ? n : 1), st));
    CK(bn.alloc(sizeof(int32_t) * (hg->p > 0 ? hg->p : 1), st));
    CK(offs.alloc(sizeof(unsigned) * 2 * (k + 1), st));
    CK(scr.alloc(sizeof(unsigned) * (scan_scratch_words((unsigned)cmax) + 8), st));
    CK(tot.alloc(sizeof(unsigned) * 2, st));
    CK(dbw.alloc(sizeof(unsigned long long) * k, st));
    CK(cudaMemsetAsync(offs.p, 0, sizeof(unsigned) * 2 * (k + 1), st));
    CK(cudaMemsetAsync(dbw.p, 0, sizeof(unsigned long long) * k, st));
    unsigned* of = offs.as<unsigned>();
    if (n) {
      k_grp_count<<<Tv, kGrpTile, 0, st>>>(n, part, nullptr, k, Tv, C.as<unsigned>());
      scan_exclusive(C.as<unsigned>(), (unsigned)k * Tv, scr.as<unsigned>(), tot.as<unsigned>(),
                     st);
      k_grp_place<<<Tv, kGrpTile, 0, st>>>(n, part, nullptr, k, Tv, C.as<unsigned>(),
                                           bv.as<int32_t>());
      k_grp_offsets<<<1, 64, 0, st>>>(C.as<unsigned>(), Tv, k, tot.as<unsigned>(), of);
      k_block_weights<<<nb(n, 256, sms * 8), 256, 0, st>>>(n, part, hg->node_w,
                                                           dbw.as<unsigned long long>());
      count_launches(5);
    }
    if (m) {
      k_net_mask<<<nb((long long)m * 32, 256, sms * 16), 256, 0, st>>>(
          m, hg->net_off, hg->pins, part, nmask.as<unsigned long long>());
      k_grp_count<<<Tn, kGrpTile, 0, st>>>(m, nullptr, nmask.as<unsigned long long>(), k, Tn,
                                           C.as<unsigned>());
      scan_exclusive(C.as<unsigned>(), (unsigned)k * Tn, scr.as<unsigned>(),
                     tot.as<unsigned>() + 1, st);
      k_grp_place<<<Tn, kGrpTile, 0, st>>>(m, nullptr, nmask.as<unsigned long long>(), k, Tn,
                                           C.as<unsigned>(), bn.as<int32_t>());
      k_grp_offsets<<<1, 64, 0, st>>>(C.as<unsigned>(), Tn, k, tot.as<unsigned>() + 1,
                                      of + (k + 1));
      count_launches(4);
    }
    std::vector<unsigned> h(2 * (k + 1));
    bw.assign(k, 0);
    CK(cudaMemcpyAsync(h.data(), of, sizeof(unsigned) * 2 * (k + 1), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(bw.data(), dbw.p, sizeof(unsigned long long) * k, cudaMemcpyDeviceToHost,
                       st));
    CK(cudaStreamSynchronize(st));
    bv_off.assign(h.begin(), h.begin() + (k + 1));
    bn_off.assign(h.begin() + (k + 1), h.end());
    return HFP_OK;
  }
};

// A block pair between region growing and the moves.
struct PairWork {
  hfp_pair_result r{};
  hfp_net* net = nullptr;
  DevBuf region;      // region vertices, ascending
  int32_t nr = 0;
  PairWork() = default;
  PairWork(const PairWork&) = delete;
  ~PairWork() {
    if (net) hfp_net_destroy(net);
  }
};

// Compaction of list[i] for flag[i] != 0 into out (list order), optionally
// with the vertex weights; returns the count (synchronises).
hfp_status compact_list(hfp_ctx* ctx, hfp_hgraph* hg, unsigned cnt, const int32_t* list,
                        unsigned* flag, unsigned* pos, int32_t* out, unsigned* wout, unsigned* scr,
                        unsigned* tot, unsigned* count) {
  cudaStream_t st = ctx->stream;
  if (cnt == 0) {
    *count = 0;
    return HFP_OK;
  }
  CK(cudaMemcpyAsync(pos, flag, sizeof(unsigned) * cnt, cudaMemcpyDeviceToDevice, st));
  scan_exclusive(pos, cnt, scr, tot, st);
  k_list_scatter<<<nb(cnt, 256, ctx->sms * 8), 256, 0, st>>>(cnt, list, flag, pos, out,
                                                                 hg->node_w, wout);
  count_launches(1);
  CK(cudaMemcpyAsync(count, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}

// Whether block-pair networks use the second construction algorithm
// (Section 6): always (mode 2), never (1), or as the paper decides (0: for
// sparse hypergraphs, |E| / |V| <= 0.5, or large nets, average size >= 100).
bool sorted_construction(const hfp_hgraph* hg, uint32_t cmode) {
  return cmode == 2 ||
         (cmode == 0 && ((long long)hg->m * 2 <= (long long)hg->n || hg->p >= 100ll * hg->m));
}

// Region of the pair (Section 6), its flow network and the pair's original
// cut on the network's nets, on the stream of ctx (the hypergraph's context
// or a helper context of it; sc belongs to that stream).  Everything but the
// flow network's own construction works on the two blocks' vertex and net
// lists.
hfp_status prepare_pair(hfp_hgraph* hg, hfp_ctx* ctx, const int32_t* part, int32_t k, int32_t bi,
                        int32_t bj, const hfp_refine_params* prm, RegionScratch& sc,
                        BlockLists& bl, PairWork& w) {
  cudaStream_t st = ctx->stream;
  const int n = hg->n, m = hg->m, sms = ctx->sms;
  hfp_pair_result* res = &w.r;
  memset(res, 0, sizeof(*res));
  res->bi = bi;
  res->bj = bj;
  (void)k;
  const int32_t* bv = bl.bv.as<int32_t>();
  const int32_t* bn = bl.bn.as<int32_t>();
  const unsigned long long* nmask = bl.nmask.as<unsigned long long>();
  const int32_t* V[2] = {bv + bl.bv_off[bi], bv + bl.bv_off[bj]};
  const unsigned nv[2] = {bl.bv_off[bi + 1] - bl.bv_off[bi], bl.bv_off[bj + 1] - bl.bv_off[bj]};
  const int32_t* Ni = bn + bl.bn_off[bi];
  const int32_t* Nj = bn + bl.bn_off[bj];
  const unsigned nni = bl.bn_off[bi + 1] - bl.bn_off[bi], nnj = bl.bn_off[bj + 1] - bl.bn_off[bj];
  int32_t* side = sc.side.as<int32_t>();
  int32_t* lev = sc.lev.as<int32_t>();
  uint8_t* inb = sc.inb.as<uint8_t>();
  for (int s = 0; s < 2; s++)
    if (nv[s]) {
      k_list_side<<<nb(nv[s], 256, sms * 8), 256, 0, st>>>(nv[s], V[s], s, side, lev, inb);
      count_launches(1);
    }
  if (nni) {
    k_level1_list<<<nb((long long)nni * 32, 256, sms * 16), 256, 0, st>>>(
        nni, Ni, nmask, bi, bj, hg->net_off, hg->pins, side, lev);
    count_launches(1);
  }
  const unsigned long long cw[2] = {bl.bw[bi], bl.bw[bj]};
  const long long half = (long long)((cw[0] + cw[1] + 1) / 2);
  const long long lim = ((long long)(100 + prm->alpha_eps_pct) * half) / 100;
  long long budget[2] = {std::max(0ll, lim - (long long)cw[1]),
                         std::max(0ll, lim - (long long)cw[0])};
  unsigned h_cnt = 0;
  for (int s = 0; s < 2; s++) {
    long long left = budget[s];
    for (int d = 1; d <= prm->delta; d++) {
      if (nv[s] == 0) break;
      k_list_flag<<<nb(nv[s], 256, sms * 8), 256, 0, st>>>(nv[s], V[s], lev, inb, d,
                                                           sc.flag.as<unsigned>());
      count_launches(1);
      hfp_status r = compact_list(ctx, hg, nv[s], V[s], sc.flag.as<unsigned>(),
                                  sc.pos.as<unsigned>(), sc.cand.as<int32_t>(), sc.wts.as<unsigned>(),
                                  sc.scr.as<unsigned>(), sc.tot.as<unsigned>(), &h_cnt);
      if (r != HFP_OK) return r;
      if (h_cnt == 0) break;
      scan_exclusive(sc.wts.as<unsigned>(), h_cnt, sc.scr.as<unsigned>(), sc.tot.as<unsigned>(),
                     st);
      CK(cudaMemsetAsync(sc.taken.p, 0, sizeof(unsigned), st));
      k_take<<<nb(h_cnt, 256, sms * 8), 256, 0, st>>>(h_cnt, sc.cand.as<int32_t>(),
                                                      sc.wts.as<unsigned>(), hg->node_w, left,
                                                      inb, sc.taken.as<unsigned>());
      count_launches(1);
      unsigned h2[2];
      CK(cudaMemcpyAsync(&h2[0], sc.taken.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(&h2[1], sc.tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (h2[0] < h_cnt) break;           // the first vertex that does not fit ends growth
      left -= (long long)h2[1];
      if (d == prm->delta) break;
      k_next_level<<<nb((long long)h_cnt * 32, 256, sms * 16), 256, 0, st>>>(
          h_cnt, sc.cand.as<int32_t>(), hg->vnet_off, hg->vnet, hg->net_off, hg->pins, side, s,
          lev, d + 1);
      count_launches(1);
    }
  }
  // region: the taken vertices of each block (ascending), merged
  unsigned rc[2] = {0, 0};
  int32_t* rv = sc.rv.as<int32_t>();
  for (int s = 0; s < 2; s++) {
    if (nv[s] == 0) continue;
    k_list_flag<<<nb(nv[s], 256, sms * 8), 256, 0, st>>>(nv[s], V[s], lev, inb, -1,
                                                         sc.flag.as<unsigned>());
    count_launches(1);
    hfp_status r = compact_list(ctx, hg, nv[s], V[s], sc.flag.as<unsigned>(),
                                sc.pos.as<unsigned>(), rv + rc[0], nullptr, sc.scr.as<unsigned>(), sc.tot.as<unsigned>(),
                                &rc[s]);
    if (r != HFP_OK) return r;
  }
  const unsigned nr = rc[0] + rc[1];
  DevBuf dist;
  CK(dist.alloc(sizeof(int32_t) * (nr > 0 ? nr : 1), st));
  CK(w.region.alloc(sizeof(int32_t) * (nr > 0 ? nr : 1), st));
  if (nr) {
    k_merge_sorted<<<nb(nr, 256, sms * 8), 256, 0, st>>>(rv, rc[0], rv + rc[0], rc[1],
                                                         w.region.as<int32_t>());
    k_region_dist<<<nb(nr, 256, sms * 8), 256, 0, st>>>(nr, w.region.as<int32_t>(), lev,
                                                        dist.as<int32_t>());
    count_launches(2);
  }
  w.nr = (int32_t)nr;
  res->region_size = (int32_t)nr;
  // Construction (Section 6): the first algorithm scans the nets of the two
  // blocks, the second sorts the region's incidences by net
  const bool sorted_build = sorted_construction(hg, ctx->construction);
  SortBuildIn sbi{};
  if (sorted_build) {
    if (hfp_status r0 = bl.build_counts(hg, part)) return r0;
    sbi = SortBuildIn{hg->vnet_off, hg->vnet, nmask, bl.noff.as<unsigned>(),
                      bl.cnt.as<unsigned>(), bi, bj};
  }
  // nets of the network (first algorithm): those of block bi, and those of
  // block bj without a pin in bi, merged into ascending order; vertices: both
  // blocks
  unsigned nj2 = 0;
  if (nnj && !sorted_build) {
    k_net_not_in<<<nb(nnj, 256, sms * 8), 256, 0, st>>>(nnj, Nj, nmask, bi,
                                                        sc.flag.as<unsigned>());
    count_launches(1);
    hfp_status r = compact_list(ctx, hg, nnj, Nj, sc.flag.as<unsigned>(),
                                sc.pos.as<unsigned>(), sc.nets2.as<int32_t>(), nullptr, sc.scr.as<unsigned>(),
                                sc.tot.as<unsigned>(), &nj2);
    if (r != HFP_OK) return r;
  }
  const unsigned nnet = sorted_build ? 0u : nni + nj2;
  if (nnet) {
    k_merge_sorted<<<nb(nnet, 256, sms * 8), 256, 0, st>>>(Ni, nni, sc.nets2.as<int32_t>(), nj2,
                                                           sc.netlist.as<int32_t>());
    count_launches(1);
  }
  if (nv[0]) CK(cudaMemcpyAsync(sc.vlist.p, V[0], sizeof(int32_t) * nv[0], cudaMemcpyDeviceToDevice, st));
  if (nv[1])
    CK(cudaMemcpyAsync(sc.vlist.as<int32_t>() + nv[0], V[1], sizeof(int32_t) * nv[1],
                       cudaMemcpyDeviceToDevice, st));
  hfp_hypergraph Hd{n, m, hg->net_off, hg->pins, hg->net_w, hg->node_w};
  hfp_status r = build_network_impl(ctx, &Hd, HFP_MEM_DEVICE, w.region.as<int32_t>(), (int32_t)nr,
                                    side, dist.as<int32_t>(), sc.netlist.as<int32_t>(),
                                    (int32_t)nnet, sc.vlist.as<int32_t>(),
                                    (int32_t)(nv[0] + nv[1]), &w.net,
                                    sorted_build ? &sbi : nullptr);
  // the two blocks' entries go back for the next pair
  for (int s = 0; s < 2; s++)
    if (nv[s]) {
      k_list_side<<<nb(nv[s], 256, sms * 8), 256, 0, st>>>(nv[s], V[s], -1, side, lev, inb);
      count_launches(1);
    }
  if (r != HFP_OK) return r;
  res->pins = w.net->d.p_pins;
  CK(cudaMemsetAsync(sc.cut.p, 0, sizeof(unsigned long long), st));
  if (w.net->d.m_nets) {
    k_pair_cut<<<nb((long long)w.net->d.m_nets * 32, 256, sms * 16), 256, 0, st>>>(
        w.net->d, sc.cut.as<unsigned long long>());
    count_launches(1);
  }
  unsigned long long hc = 0;
  CK(cudaMemcpyAsync(&hc, sc.cut.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  res->original_cut = (int64_t)hc;
  return HFP_OK;
}

// Prepares the pairs of a batched round into works (one entry per pair, in
// pair order).  With prep_streams > 1 the pairs go to that many host
// threads, each with a helper context (stream, pinned staging) and region
// scratch of its own, which take the next pair from a shared counter, so that
// the host round trips of different pairs overlap.  A network does not
// depend on which thread built it.  Once every helper stream has finished,
// the networks move to the hypergraph's context.
hfp_status prepare_pairs(hfp_hgraph* hg, const int32_t* part, int32_t k,
                         const hfp_refine_params* prm,
                         const std::vector<std::pair<int, int>>& pairs, RegionScratch& sc,
                         BlockLists& bl, std::deque<PairWork>& works) {
  hfp_ctx* ctx = hg->ctx;
  const int n = (int)pairs.size();
  const int base = (int)works.size();
  for (int t = 0; t < n; t++) works.emplace_back();
  const int W = std::min<int>((int)ctx->prep_streams, n);
  if (W <= 1) {
    for (int t = 0; t < n; t++) {
      hfp_status s = prepare_pair(hg, ctx, part, k, pairs[t].first, pairs[t].second, prm, sc, bl,
                                  works[base + t]);
      if (s != HFP_OK) return s;
    }
    return HFP_OK;
  }
  if (sorted_construction(hg, ctx->construction))
    if (hfp_status s = bl.build_counts(hg, part)) return s;
  // the block lists and the partition are complete before the helpers start
  CK(cudaStreamSynchronize(ctx->stream));
  while ((int)hg->prep.size() < W) {
    hfp_ctx* c = nullptr;
    if (hfp_status s = ctx_fork(ctx, &c)) return s;
    hg->prep.push_back(c);
  }
  for (int w = 0; w < W; w++) ctx_copy_tuning(hg->prep[w], ctx);
  std::atomic<int> next{0}, stop{0};
  std::vector<hfp_status> status(W, HFP_OK);
  std::vector<std::string> msg(W);
  auto body = [&](int w) {
    hfp_ctx* c = hg->prep[w];
    hfp_status s = cudaSetDevice(c->device) == cudaSuccess
                       ? HFP_OK
                       : fail(HFP_ERR_CUDA, "pair preparation: cudaSetDevice failed");
    {
      RegionScratch wsc;
      if (s == HFP_OK) s = wsc.alloc(hg, c->stream);
      while (s == HFP_OK && !stop.load()) {
        const int t = next.fetch_add(1);
        if (t >= n) break;
        s = prepare_pair(hg, c, part, k, pairs[t].first, pairs[t].second, prm, wsc, bl,
                         works[base + t]);
      }
    }
    const cudaError_t e = cudaStreamSynchronize(c->stream);
    if (s == HFP_OK && e != cudaSuccess)
      s = fail(HFP_ERR_CUDA, "pair preparation: %s", cudaGetErrorString(e));
    if (s != HFP_OK) {
      stop.store(1);
      status[w] = s;
      msg[w] = hfp_last_error();
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < W; w++) th.emplace_back(body, w);
  body(0);
  for (auto& x : th) x.join();
  for (int t = 0; t < n; t++) {
    net_rehome(works[base + t].net, ctx);
    works[base + t].region.st = ctx->stream;
  }
  for (int w = 0; w < W; w++)
    if (status[w] != HFP_OK) {
      set_last_error(msg[w].c_str());
      return status[w];
    }
  return HFP_OK;
}

// FlowCutter parameters of a pair: the k-way bound L and the original cut as
// flow bound (Section 8.3, "Flow Value").
hfp_fc_params pair_fc_params(hfp_hgraph* hg, int32_t k, const hfp_refine_params* prm,
                             const PairWork& w) {
  hfp_fc_params fp{};
  fp.max_block_weight = ((100 + prm->eps_pct) * ((hg->total_w + k - 1) / k)) / 100;
  fp.flow_bound = w.r.original_cut;
  fp.seed = prm->seed;
  fp.max_iterations = 0;
  return fp;
}

// FlowCutter outcome -> result fields and the moves (region order) against
// the partition the pair was prepared with.  The network is released.
hfp_status finish_pair(hfp_hgraph* hg, const int32_t* part, hfp_status fc, const hfp_fc_result& fr,
                       RegionScratch& sc, PairWork& w, DevBuf& moves_dev) {
  hfp_ctx* ctx = hg->ctx;
  cudaStream_t st = ctx->stream;
  const int sms = ctx->sms;
  hfp_pair_result* res = &w.r;
  res->status = fc;
  res->flow = fr.flow;
  res->iterations = fr.iterations;
  res->device_us = fr.device_us;
  if (fc == HFP_NO_BALANCED_CUT || fc == HFP_ABORTED_WORSE) {
    hfp_net_destroy(w.net);
    w.net = nullptr;
    set_last_error("");
    return HFP_OK;
  }
  if (fc != HFP_OK) return fc;
  res->delta_exp = res->original_cut - fr.flow;
  const unsigned nr = (unsigned)w.nr;
  unsigned nm = 0;
  if (nr) {
    DevBuf fin, mflag, mpos;
    CK(fin.alloc(nr, st));
    CK(mflag.alloc(sizeof(unsigned) * nr, st));
    CK(mpos.alloc(sizeof(unsigned) * nr, st));
    launch_region_side(w.net->d, fr.result_side, (int32_t)nr, fin.as<uint8_t>(), sms, st);
    k_move_flags<<<nb(nr, 256, sms * 8), 256, 0, st>>>(nr, w.region.as<int32_t>(), part, res->bi,
                                                       fin.as<uint8_t>(), mflag.as<unsigned>());
    count_launches(1);
    CK(cudaMemcpyAsync(mpos.p, mflag.p, sizeof(unsigned) * nr, cudaMemcpyDeviceToDevice, st));
    scan_exclusive(mpos.as<unsigned>(), nr, sc.scr.as<unsigned>(), sc.tot.as<unsigned>(), st);
    CK(cudaMemcpyAsync(&nm, sc.tot.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(moves_dev.alloc(sizeof(int32_t) * 3 * (nm > 0 ? nm : 1), st));
    k_move_fill<<<nb(nr, 256, sms * 8), 256, 0, st>>>(nr, w.region.as<int32_t>(), fin.as<uint8_t>(),
                                                      mflag.as<unsigned>(), mpos.as<unsigned>(),
                                                      res->bi, res->bj, moves_dev.as<int32_t>());
    count_launches(1);
  }
  res->n_moves = (int32_t)nm;
  hfp_net_destroy(w.net);
  w.net = nullptr;
  return HFP_OK;
}

// One pair, one problem per launch sequence: region, network, FlowCutter
// (hfp_flowcutter), moves.
hfp_status refine_pair(hfp_hgraph* hg, const int32_t* part, int32_t k, int32_t bi, int32_t bj,
                       const hfp_refine_params* prm, RegionScratch& sc, BlockLists& bl,
                       DevBuf& moves_dev, hfp_pair_result* res) {
  PairWork w;
  hfp_status s = prepare_pair(hg, hg->ctx, part, k, bi, bj, prm, sc, bl, w);
  if (s != HFP_OK) return s;
  const hfp_fc_params fp = pair_fc_params(hg, k, prm, w);
  hfp_fc_result fr{};
  const hfp_status fc = hfp_flowcutter(w.net, &fp, nullptr, nullptr, nullptr, 0, &fr);
  s = finish_pair(hg, part, fc, fr, sc, w, moves_dev);
  *res = w.r;
  return s;
}

}  // namespace

HFP_API hfp_status hfp_refine_block_pair(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                         int32_t bi, int32_t bj, const hfp_refine_params* prm,
                                         int32_t* moves, int32_t cap, hfp_pair_result* res) {
  if (!hg || !part || !prm || !res) return fail(HFP_ERR_INVALID, "NULL argument");
  if (k < 2 || k > 64 || bi < 0 || bj < 0 || bi >= k || bj >= k || bi == bj || prm->delta < 1)
    return fail(HFP_ERR_INVALID, "bad block pair");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  RegionScratch sc;
  if ((s = sc.alloc(hg, hg->ctx->stream)) != HFP_OK) return s;
  BlockLists bl;
  if ((s = bl.build(hg, part, k)) != HFP_OK) return s;
  DevBuf mv;
  if ((s = refine_pair(hg, part, k, bi, bj, prm, sc, bl, mv, res)) != HFP_OK) return s;
  if (moves && res->n_moves > 0) {
    const int32_t c = res->n_moves < cap ? res->n_moves : cap;
    if (c > 0)
      CK(cudaMemcpyAsync(moves, mv.p, sizeof(int32_t) * 3 * c, cudaMemcpyDeviceToHost,
                         hg->ctx->stream));
    CK(cudaStreamSynchronize(hg->ctx->stream));
    if (res->n_moves > cap)
      return fail(HFP_ERR_BUFFER_TOO_SMALL, "moves needs %d entries", res->n_moves);
  }
  return HFP_OK;
}

HFP_API hfp_status hfp_connectivity(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                    int64_t* value) {
  if (!hg || !part || !value || k < 1 || k > 64) return fail(HFP_ERR_INVALID, "bad arguments");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  cudaStream_t st = hg->ctx->stream;
  DevBuf out;
  CK(out.alloc(sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(out.p, 0, sizeof(unsigned long long), st));
  if (hg->m) {
    k_connectivity<<<nb((long long)hg->m * 32, 256, hg->ctx->sms * 16), 256, 0, st>>>(
        hg->m, hg->net_off, hg->pins, hg->net_w, part, out.as<unsigned long long>(), nullptr,
        nullptr, k);
    count_launches(1);
  }
  unsigned long long h = 0;
  CK(cudaMemcpyAsync(&h, out.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  *value = (int64_t)h;
  return HFP_OK;
}

namespace {

// Pairs of adjacent blocks (quotient graph, Section 5) in ascending (i, j);
// fills stats->connectivity_before and ->pairs_skipped.
hfp_status round_pairs(hfp_hgraph* hg, const int32_t* part, int32_t k, const float* pair_scores,
                       float min_score, hfp_round_stats* stats,
                       std::vector<std::pair<int, int>>& pairs,
                       std::vector<long long>* pair_nets = nullptr) {
  cudaStream_t st = hg->ctx->stream;
  const int m = hg->m, sms = hg->ctx->sms;
  DevBuf conn, qn, qw;
  CK(conn.alloc(sizeof(unsigned long long), st));
  CK(qn.alloc(sizeof(unsigned long long) * k * k, st));
  CK(qw.alloc(sizeof(unsigned long long) * k * k, st));
  CK(cudaMemsetAsync(conn.p, 0, sizeof(unsigned long long), st));
  CK(cudaMemsetAsync(qn.p, 0, sizeof(unsigned long long) * k * k, st));
  CK(cudaMemsetAsync(qw.p, 0, sizeof(unsigned long long) * k * k, st));
  if (m) {
    k_connectivity<<<nb((long long)m * 32, 256, sms * 16), 256, 0, st>>>(
        m, hg->net_off, hg->pins, hg->net_w, part, conn.as<unsigned long long>(),
        qn.as<unsigned long long>(), qw.as<unsigned long long>(), k);
    count_launches(1);
  }
  std::vector<unsigned long long> hq((size_t)k * k);
  unsigned long long c0 = 0;
  CK(cudaMemcpyAsync(hq.data(), qn.p, sizeof(unsigned long long) * k * k, cudaMemcpyDeviceToHost,
                     st));
  CK(cudaMemcpyAsync(&c0, conn.p, sizeof(c0), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  stats->connectivity_before = (int64_t)c0;
  for (int i = 0; i < k; i++)
    for (int j = i + 1; j < k; j++) {
      if (hq[(size_t)i * k + j] == 0) continue;
      if (pair_scores && pair_scores[(size_t)i * k + j] < min_score) {
        stats->pairs_skipped++;
        continue;
      }
      pairs.emplace_back(i, j);
      if (pair_nets) pair_nets->push_back((long long)hq[(size_t)i * k + j]);
    }
  return HFP_OK;
}

struct Item {
  hfp_pair_result r;
  DevBuf mv;
};

// Host wall-clock milliseconds since t0; the caller synchronises first.
inline float ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<float, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// Refines every pair against the same partition: one FlowCutter per launch
// sequence (plain) or all FlowCutter problems in one batched launch.
hfp_status refine_pairs(hfp_hgraph* hg, const int32_t* part, int32_t k,
                        const hfp_refine_params* prm, const std::vector<std::pair<int, int>>& pairs,
                        bool batched, int32_t group_ctas, std::deque<Item>& items,
                        float* flow_ms, hfp_round_stats* stats) {
  RegionScratch sc;
  hfp_status s = sc.alloc(hg, hg->ctx->stream);
  if (s != HFP_OK) return s;
  auto t0 = std::chrono::steady_clock::now();
  BlockLists bl;
  if ((s = bl.build(hg, part, k)) != HFP_OK) return s;
  if (!batched) {
    for (const auto& pr : pairs) {
      items.emplace_back();
      if ((s = refine_pair(hg, part, k, pr.first, pr.second, prm, sc, bl, items.back().mv,
                           &items.back().r)) != HFP_OK)
        return s;
    }
    CK(cudaStreamSynchronize(hg->ctx->stream));
    stats->ms_prepare = ms_since(t0);
    return HFP_OK;
  }
  std::deque<PairWork> works;
  if ((s = prepare_pairs(hg, part, k, prm, pairs, sc, bl, works)) != HFP_OK) return s;
  CK(cudaStreamSynchronize(hg->ctx->stream));
  stats->ms_prepare = ms_since(t0);
  t0 = std::chrono::steady_clock::now();
  const int n = (int)works.size();
  std::vector<BatchItem> bi(n);
  for (int t = 0; t < n; t++) {
    bi[t].net = works[t].net;
    bi[t].params = pair_fc_params(hg, k, prm, works[t]);
  }
  const int G = group_ctas > 0 ? group_ctas : hg->tuned_group;
  if ((s = run_fc_batch(hg->ctx, bi.data(), n, G, flow_ms,
                        hg->tuned_engine ? &hg->tuned : nullptr)) != HFP_OK)
    return s;
  stats->ms_flow = ms_since(t0);
  t0 = std::chrono::steady_clock::now();
  for (int t = 0; t < n; t++) {
    items.emplace_back();
    works[t].r.group_ctas = bi[t].group_ctas;
    s = finish_pair(hg, part, bi[t].status, bi[t].result, sc, works[t], items.back().mv);
    items.back().r = works[t].r;
    if (s != HFP_OK) return s;
  }
  CK(cudaStreamSynchronize(hg->ctx->stream));
  stats->ms_finish = ms_since(t0);
  return HFP_OK;
}

// Algorithm 1's apply step (Section 5, "Apply Moves") on the refined pairs.
hfp_status apply_round(hfp_hgraph* hg, int32_t* part, int32_t k, const hfp_refine_params* prm,
                       std::deque<Item>& items, hfp_round_stats* stats) {
  hfp_ctx* ctx = hg->ctx;
  cudaStream_t st = ctx->stream;
  const int n = hg->n, m = hg->m, sms = ctx->sms;
  stats->pairs = (int32_t)items.size();
  // apply in descending Delta_exp, ties ascending (i, j)
  std::vector<int> order;
  for (int t = 0; t < (int)items.size(); t++) {
    const hfp_pair_result& r = items[t].r;
    if (r.status == HFP_OK && r.delta_exp >= 0 && r.n_moves > 0) order.push_back(t);
    if (r.status == HFP_OK && r.delta_exp > 0) stats->pairs_improved++;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const hfp_pair_result &x = items[a].r, &y = items[b].r;
    if (x.delta_exp != y.delta_exp) return x.delta_exp > y.delta_exp;
    if (x.bi != y.bi) return x.bi < y.bi;
    return x.bj < y.bj;
  });
  const long long L = ((100 + prm->eps_pct) * ((hg->total_w + k - 1) / k)) / 100;
  DevBuf bw, dw, valid, nvalid, gain, moved_to, moved_stamp, net_stamp;
  CK(bw.alloc(sizeof(unsigned long long) * k, st));
  CK(dw.alloc(sizeof(long long) * k, st));
  CK(nvalid.alloc(sizeof(unsigned), st));
  CK(gain.alloc(sizeof(long long), st));
  CK(moved_to.alloc(sizeof(int32_t) * (n > 0 ? n : 1), st));
  CK(moved_stamp.alloc(sizeof(unsigned) * (n > 0 ? n : 1), st));
  CK(net_stamp.alloc(sizeof(unsigned) * (m > 0 ? m : 1), st));
  CK(cudaMemsetAsync(bw.p, 0, sizeof(unsigned long long) * k, st));
  CK(cudaMemsetAsync(moved_stamp.p, 0, sizeof(unsigned) * (n > 0 ? n : 1), st));
  CK(cudaMemsetAsync(net_stamp.p, 0, sizeof(unsigned) * (m > 0 ? m : 1), st));
  if (n) {
    k_block_weights<<<nb(n, 256, sms * 8), 256, 0, st>>>(n, part, hg->node_w,
                                                         bw.as<unsigned long long>());
    count_launches(1);
  }
  std::vector<long long> hbw(k), hdw(k);
  CK(cudaMemcpyAsync(hbw.data(), bw.p, sizeof(long long) * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  unsigned epoch = 0;
  for (int t : order) {
    Item& it = items[t];
    const unsigned cnt = (unsigned)it.r.n_moves;
    epoch++;
    CK(valid.alloc(cnt, st));
    CK(cudaMemsetAsync(dw.p, 0, sizeof(long long) * k, st));
    CK(cudaMemsetAsync(nvalid.p, 0, sizeof(unsigned), st));
    CK(cudaMemsetAsync(gain.p, 0, sizeof(long long), st));
    k_apply_check<<<nb(cnt, 256, sms * 8), 256, 0, st>>>(
        cnt, it.mv.as<int32_t>(), part, hg->node_w, valid.as<uint8_t>(), dw.as<long long>(),
        nvalid.as<unsigned>(), moved_to.as<int32_t>(), epoch, moved_stamp.as<unsigned>());
    count_launches(1);
    unsigned hv = 0;
    CK(cudaMemcpyAsync(hdw.data(), dw.p, sizeof(long long) * k, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hv, nvalid.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    bool ok = hv > 0;
    for (int b = 0; b < k && ok; b++)
      if (hdw[b] > 0 && hbw[b] + hdw[b] > L) ok = false;
    long long g = 0;
    if (ok) {
      k_apply_gain<<<nb((long long)cnt * 32, 256, sms * 16), 256, 0, st>>>(
          cnt, it.mv.as<int32_t>(), valid.as<uint8_t>(), hg->vnet_off, hg->vnet, hg->net_off,
          hg->pins, hg->net_w, part, moved_to.as<int32_t>(), moved_stamp.as<unsigned>(),
          net_stamp.as<unsigned>(), epoch, it.r.bi, it.r.bj, gain.as<long long>());
      count_launches(1);
      CK(cudaMemcpyAsync(&g, gain.p, sizeof(g), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (g >= 0) {
        k_apply_commit<<<nb(cnt, 256, sms * 8), 256, 0, st>>>(cnt, it.mv.as<int32_t>(),
                                                             valid.as<uint8_t>(), part);
        count_launches(1);
        for (int b = 0; b < k; b++) hbw[b] += hdw[b];
        it.r.applied = 1;
        it.r.gain = g;
        stats->gain += g;
        stats->pairs_applied++;
        stats->moves_applied += hv;
      }
    }
    it.r.valid_moves = (int32_t)hv;
    if (valid.p) {
      cudaFreeAsync(valid.p, st);
      valid.p = nullptr;
    }
  }
  CK(cudaStreamSynchronize(st));
  stats->connectivity_after = stats->connectivity_before - stats->gain;
  return HFP_OK;
}

hfp_status round_impl(hfp_hgraph* hg, int32_t* part, int32_t k, const hfp_refine_params* prm,
                      const float* pair_scores, float min_score, hfp_round_stats* stats,
                      hfp_pair_result* pairs, int32_t cap, int32_t* n_pairs, bool batched,
                      int32_t group_ctas, float* flow_ms) {
  if (!hg || !part || !prm || !stats) return fail(HFP_ERR_INVALID, "NULL argument");
  if (k < 2 || k > 64) return fail(HFP_ERR_INVALID, "k must be in [2, 64]");
  if (prm->delta < 1) return fail(HFP_ERR_INVALID, "delta must be positive");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  memset(stats, 0, sizeof(*stats));
  std::vector<std::pair<int, int>> pl;
  auto t0 = std::chrono::steady_clock::now();
  if ((s = round_pairs(hg, part, k, pair_scores, min_score, stats, pl)) != HFP_OK) return s;
  stats->ms_pairs = ms_since(t0);
  std::deque<Item> items;
  if ((s = refine_pairs(hg, part, k, prm, pl, batched, group_ctas, items, flow_ms, stats)) !=
      HFP_OK)
    return s;
  t0 = std::chrono::steady_clock::now();
  if ((s = apply_round(hg, part, k, prm, items, stats)) != HFP_OK) return s;
  stats->ms_apply = ms_since(t0);
  if (n_pairs) *n_pairs = (int32_t)items.size();
  if (pairs)
    for (int t = 0; t < (int)items.size() && t < cap; t++) pairs[t] = items[t].r;
  return HFP_OK;
}

}  // namespace

HFP_API hfp_status hfp_refine_round(hfp_hgraph* hg, int32_t* part, int32_t k,
                                    const hfp_refine_params* prm, const float* pair_scores,
                                    float min_score, hfp_round_stats* stats,
                                    hfp_pair_result* pairs, int32_t cap, int32_t* n_pairs) {
  return round_impl(hg, part, k, prm, pair_scores, min_score, stats, pairs, cap, n_pairs, false,
                    0, nullptr);
}

HFP_API hfp_status hfp_refine_round_batched(hfp_hgraph* hg, int32_t* part, int32_t k,
                                            const hfp_refine_params* prm,
                                            const float* pair_scores, float min_score,
                                            int32_t group_ctas, hfp_round_stats* stats,
                                            hfp_pair_result* pairs, int32_t cap,
                                            int32_t* n_pairs, float* flowcutter_ms) {
  return round_impl(hg, part, k, prm, pair_scores, min_score, stats, pairs, cap, n_pairs, true,
                    group_ctas, flowcutter_ms);
}

HFP_API hfp_status hfp_autotune_round(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                      const hfp_refine_params* prm, const int32_t* candidates,
                                      int32_t n_candidates, float* ms, int32_t* best) {
  if (!hg || !part || !prm || !candidates || n_candidates <= 0)
    return fail(HFP_ERR_INVALID, "bad arguments");
  if (k < 2 || k > 64 || prm->delta < 1) return fail(HFP_ERR_INVALID, "bad k or delta");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  int grid = 0;
  if ((s = batch_grid(hg->ctx, &grid)) != HFP_OK) return s;
  for (int c = 0; c < n_candidates; c++)
    if (candidates[c] < 1 || candidates[c] > grid)
      return fail(HFP_ERR_INVALID, "candidate %d: group size %d outside [1, %d]", c,
                  candidates[c], grid);
  hfp_round_stats st{};
  std::vector<std::pair<int, int>> pl;
  if ((s = round_pairs(hg, part, k, nullptr, 0.f, &st, pl)) != HFP_OK) return s;
  RegionScratch sc;
  if ((s = sc.alloc(hg, hg->ctx->stream)) != HFP_OK) return s;
  BlockLists bl;
  if ((s = bl.build(hg, part, k)) != HFP_OK) return s;
  float best_ms = 0.f;
  int best_g = 0;
  for (int c = 0; c < n_candidates; c++) {
    // the same networks, rebuilt for every candidate
    std::deque<PairWork> works;
    if ((s = prepare_pairs(hg, part, k, prm, pl, sc, bl, works)) != HFP_OK) return s;
    const int n = (int)works.size();
    std::vector<BatchItem> bi(n);
    for (int t = 0; t < n; t++) {
      bi[t].net = works[t].net;
      bi[t].params = pair_fc_params(hg, k, prm, works[t]);
    }
    float t_ms = 0.f;
    if ((s = run_fc_batch(hg->ctx, bi.data(), n, candidates[c], &t_ms)) != HFP_OK) return s;
    if (ms) ms[c] = t_ms;
    if (c == 0 || t_ms < best_ms) {
      best_ms = t_ms;
      best_g = candidates[c];
    }
  }
  hg->tuned_group = best_g;
  if (best) *best = best_g;
  return HFP_OK;
}

// Engine knobs of the batched launch tried by hfp_autotune_round_engine, one
// knob after the other (the best value of a knob is kept for the next):
// global-relabel work, the stall rule of incremental flows, the CTA-alone
// round thresholds, the round form.
namespace {
struct KnobTry {
  int knob;        // 0 gr_work_x100, 1 stall_rounds_pierce, 2 tail_enter/exit, 3 fused rounds
  unsigned a, b;
};
const KnobTry kKnobTries[] = {{0, 100, 0}, {0, 200, 0}, {0, 400, 0},
                              {1, 0, 0},   {1, 30, 0},  {1, 100, 0},
                              {2, 64, 192}, {2, 16, 64}, {2, 256, 768},
                              {3, 1, 0},   {3, 0, 0}};
void apply_knob(BatchTune& t, const KnobTry& k) {
  switch (k.knob) {
    case 0: t.gr_work_x100 = k.a; break;
    case 1: t.P.stall_rounds_pierce = k.a; break;
    case 2: t.P.tail_enter = k.a; t.P.tail_exit = k.b; break;
    default: t.P.fused_rounds = k.a; break;
  }
}
}  // namespace

HFP_API hfp_status hfp_autotune_round_engine(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                             const hfp_refine_params* prm, int32_t group_ctas,
                                             float* ms, int32_t cap, int32_t* n_tried,
                                             hfp_tuning* chosen) {
  if (!hg || !part || !prm || !n_tried || (cap > 0 && !ms)) return fail(HFP_ERR_INVALID, "bad arguments");
  if (k < 2 || k > 64 || prm->delta < 1) return fail(HFP_ERR_INVALID, "bad k or delta");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  hfp_ctx* ctx = hg->ctx;
  hfp_round_stats st{};
  std::vector<std::pair<int, int>> pl;
  if ((s = round_pairs(hg, part, k, nullptr, 0.f, &st, pl)) != HFP_OK) return s;
  RegionScratch sc;
  if ((s = sc.alloc(hg, hg->ctx->stream)) != HFP_OK) return s;
  BlockLists bl;
  if ((s = bl.build(hg, part, k)) != HFP_OK) return s;
  const int G = group_ctas > 0 ? group_ctas : hg->tuned_group;
  // start from the context's knobs of batched launches
  BatchTune best{ctx->params, ctx->batch_gr_work_x100};
  best.P.fused_rounds = ctx->batch_fused_rounds;
  best.P.async_gr = ctx->batch_async_gr;
  best.P.stall_rounds_pierce = ctx->batch_stall_rounds_pierce;
  float best_ms = -1.f;
  int tried = 0;
  const int nk = (int)(sizeof(kKnobTries) / sizeof(kKnobTries[0]));
  for (int t = 0; t < nk; t++) {
    BatchTune cand = best;
    apply_knob(cand, kKnobTries[t]);
    // the same networks, rebuilt for every try
    std::deque<PairWork> works;
    if ((s = prepare_pairs(hg, part, k, prm, pl, sc, bl, works)) != HFP_OK) return s;
    const int n = (int)works.size();
    std::vector<BatchItem> bi(n);
    for (int q = 0; q < n; q++) {
      bi[q].net = works[q].net;
      bi[q].params = pair_fc_params(hg, k, prm, works[q]);
    }
    float t_ms = 0.f;
    if ((s = run_fc_batch(ctx, bi.data(), n, G, &t_ms, &cand)) != HFP_OK) return s;
    if (tried < cap) ms[tried] = t_ms;
    tried++;
    if (best_ms < 0.f || t_ms < best_ms) {
      best_ms = t_ms;
      best = cand;
    }
  }
  hg->tuned = best;
  hg->tuned_engine = true;
  *n_tried = tried;
  if (chosen) {
    if ((s = hfp_ctx_get_tuning(ctx, chosen)) != HFP_OK) return s;
    chosen->batch_gr_work_x100 = best.gr_work_x100;
    chosen->batch_stall_rounds_pierce = best.P.stall_rounds_pierce;
    chosen->tail_enter = best.P.tail_enter;
    chosen->tail_exit = best.P.tail_exit;
    chosen->batch_fused_rounds = best.P.fused_rounds;
  }
  return HFP_OK;
}

// ---------------------------------------------------------------------------
// The round in three calls, for callers that split the block pairs of a round
// across processes (one GPU each): pairs, refinement of a subset, apply step.

HFP_API hfp_status hfp_round_pairs(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                   const float* pair_scores, float min_score, int32_t* pairs,
                                   int64_t* pair_nets, int32_t cap, int32_t* n_pairs,
                                   int64_t* connectivity) {
  if (!hg || !part || !n_pairs || (cap > 0 && !pairs)) return fail(HFP_ERR_INVALID, "NULL argument");
  if (k < 2 || k > 64) return fail(HFP_ERR_INVALID, "k must be in [2, 64]");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  hfp_round_stats st{};
  std::vector<std::pair<int, int>> pl;
  std::vector<long long> nets;
  if ((s = round_pairs(hg, part, k, pair_scores, min_score, &st, pl, &nets)) != HFP_OK) return s;
  *n_pairs = (int32_t)pl.size();
  if (connectivity) *connectivity = st.connectivity_before;
  if ((int64_t)pl.size() > cap)
    return fail(HFP_ERR_BUFFER_TOO_SMALL, "%zu pairs, capacity %d", pl.size(), cap);
  for (size_t t = 0; t < pl.size(); t++) {
    pairs[2 * t] = pl[t].first;
    pairs[2 * t + 1] = pl[t].second;
    if (pair_nets) pair_nets[t] = nets[t];
  }
  return HFP_OK;
}

HFP_API hfp_status hfp_refine_pairs_batched(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                            const hfp_refine_params* prm, const int32_t* pairs,
                                            int32_t n, int32_t group_ctas,
                                            hfp_pair_result* results, int32_t* moves,
                                            int64_t move_cap, int64_t* move_off,
                                            float* flowcutter_ms) {
  if (!hg || !part || !prm || n < 0 || (n > 0 && (!pairs || !results)) || !move_off ||
      (move_cap > 0 && !moves))
    return fail(HFP_ERR_INVALID, "NULL argument");
  if (k < 2 || k > 64) return fail(HFP_ERR_INVALID, "k must be in [2, 64]");
  if (prm->delta < 1) return fail(HFP_ERR_INVALID, "delta must be positive");
  std::vector<std::pair<int, int>> pl;
  for (int32_t t = 0; t < n; t++) {
    const int32_t i = pairs[2 * t], j = pairs[2 * t + 1];
    if (i < 0 || j <= i || j >= k) return fail(HFP_ERR_INVALID, "pair %d: (%d, %d)", t, i, j);
    for (const auto& q : pl)
      if (q.first == i && q.second == j) return fail(HFP_ERR_INVALID, "pair (%d, %d) repeats", i, j);
    pl.emplace_back(i, j);
  }
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  if (flowcutter_ms) *flowcutter_ms = 0.f;
  move_off[0] = 0;
  if (n == 0) return HFP_OK;
  std::deque<Item> items;
  hfp_round_stats st{};
  if ((s = refine_pairs(hg, part, k, prm, pl, true, group_ctas, items, flowcutter_ms, &st)) !=
      HFP_OK)
    return s;
  for (int32_t t = 0; t < n; t++) {
    results[t] = items[t].r;
    move_off[t + 1] = move_off[t] + items[t].r.n_moves;
  }
  if (move_off[n] > move_cap)
    return fail(HFP_ERR_BUFFER_TOO_SMALL, "%lld moves, capacity %lld", (long long)move_off[n],
                (long long)move_cap);
  cudaStream_t st_ = hg->ctx->stream;
  for (int32_t t = 0; t < n; t++)
    if (items[t].r.n_moves > 0)
      CK(cudaMemcpyAsync(moves + 3 * move_off[t], items[t].mv.p,
                         sizeof(int32_t) * 3 * (size_t)items[t].r.n_moves, cudaMemcpyDeviceToHost,
                         st_));
  CK(cudaStreamSynchronize(st_));
  return HFP_OK;
}

HFP_API hfp_status hfp_apply_moves(hfp_hgraph* hg, int32_t* part, int32_t k,
                                   const hfp_refine_params* prm, hfp_pair_result* results,
                                   const int32_t* moves, const int64_t* move_off, int32_t n,
                                   hfp_round_stats* stats) {
  if (!hg || !part || !prm || !stats || n < 0 || (n > 0 && (!results || !move_off)))
    return fail(HFP_ERR_INVALID, "NULL argument");
  if (k < 2 || k > 64) return fail(HFP_ERR_INVALID, "k must be in [2, 64]");
  hfp_status s = hg_set_device(hg);
  if (s != HFP_OK) return s;
  memset(stats, 0, sizeof(*stats));
  int64_t c0 = 0;
  if ((s = hfp_connectivity(hg, part, k, &c0)) != HFP_OK) return s;
  stats->connectivity_before = c0;
  cudaStream_t st = hg->ctx->stream;
  std::deque<Item> items;
  for (int32_t t = 0; t < n; t++) {
    const hfp_pair_result& r = results[t];
    if (r.bi < 0 || r.bj <= r.bi || r.bj >= k) return fail(HFP_ERR_INVALID, "result %d: bad pair", t);
    if (move_off[t + 1] - move_off[t] != r.n_moves || r.n_moves < 0)
      return fail(HFP_ERR_INVALID, "result %d: %d moves, offsets give %lld", t, r.n_moves,
                  (long long)(move_off[t + 1] - move_off[t]));
    items.emplace_back();
    items.back().r = r;
    if (r.n_moves > 0) {
      if (!moves) return fail(HFP_ERR_INVALID, "moves is NULL");
      for (int64_t x = move_off[t]; x < move_off[t + 1]; x++) {
        const int32_t v = moves[3 * x], from = moves[3 * x + 1], to = moves[3 * x + 2];
        if (v < 0 || v >= hg->n || (from != r.bi && from != r.bj) || (to != r.bi && to != r.bj) ||
            from == to)
          return fail(HFP_ERR_INVALID, "result %d: bad move (%d, %d, %d)", t, v, from, to);
      }
      CK(items.back().mv.alloc(sizeof(int32_t) * 3 * (size_t)r.n_moves, st));
      CK(cudaMemcpyAsync(items.back().mv.p, moves + 3 * move_off[t],
                         sizeof(int32_t) * 3 * (size_t)r.n_moves, cudaMemcpyHostToDevice, st));
    }
  }
  auto t0 = std::chrono::steady_clock::now();
  if ((s = apply_round(hg, part, k, prm, items, stats)) != HFP_OK) return s;
  stats->ms_apply = ms_since(t0);
  for (int32_t t = 0; t < n; t++) results[t] = items[t].r;
  return HFP_OK;
}
