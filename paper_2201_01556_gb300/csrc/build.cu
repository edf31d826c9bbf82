// Flow network construction on the device (Section 6, "Construction
// Algorithms", first algorithm: a scan over the nets of H with prefix sums to
// place the pin lists, as in the paper's parallel version).
//
// Pass 1 (warp per net): count region pins, note whether the net has a pin
//   outside B on side 0 (adds s) / side 1 (adds t), decide whether it stays
//   (>= 2 pins, not both s and t), and mark region pins of nets with pins on
//   both sides (distance 1 from the original cut).
// Scans: kept-net index, pin offsets, positions in the incidence lists of s
//   and t.
// Pass 2 (warp per kept net): copy region pins in H's order by ballot
//   compaction, then s, then t; the s / t incidences go straight to their
//   scanned positions.
// Incidence of region vertices: count, scan, scatter, then a per-vertex rank
//   sort by pin slot so every list is in ascending slot order (deterministic).
#include <utility>

#include "kernels.cuh"

namespace hfp {

constexpr unsigned FULLB = 0xffffffffu;

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (three passes: tile sums, scan of tile sums, add)
constexpr int kScanThreads = 512;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned* total) {
  __shared__ unsigned warp_tot[kScanThreads / 32];
  const unsigned lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned t = __shfl_up_sync(FULLB, x, o);
    if ((int)lane >= o) x += t;
  }
  if (lane == 31) warp_tot[wid] = x;
  __syncthreads();
  if (wid == 0) {
    unsigned w = lane < (blockDim.x >> 5) ? warp_tot[lane] : 0;
    unsigned y = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned t = __shfl_up_sync(FULLB, y, o);
      if ((int)lane >= o) y += t;
    }
    if (lane < (blockDim.x >> 5)) warp_tot[lane] = y - w;
    if (lane == (blockDim.x >> 5) - 1) *total = y;
  }
  __syncthreads();
  unsigned r = x - v + warp_tot[wid];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(unsigned* a, unsigned n, unsigned* tile_sums) {
  __shared__ unsigned tot;
  unsigned base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
  unsigned v[kScanItems], s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    v[k] = (base + k < n) ? a[base + k] : 0;
    s += v[k];
  }
  unsigned off = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    if (base + k < n) a[base + k] = off;
    off += v[k];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(unsigned* sums, unsigned ntiles, unsigned* total) {
  __shared__ unsigned tot;
  unsigned carry = 0;
  for (unsigned b = 0; b < ntiles; b += kScanThreads) {
    unsigned i = b + threadIdx.x;
    unsigned v = i < ntiles ? sums[i] : 0;
    unsigned off = block_excl_scan(v, &tot);
    if (i < ntiles) sums[i] = off + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

__global__ void k_scan_add(unsigned* a, unsigned n, const unsigned* sums) {
  unsigned add = sums[blockIdx.x];
  unsigned base = blockIdx.x * kScanTile;
  for (unsigned k = threadIdx.x; k < kScanTile; k += blockDim.x)
    if (base + k < n) a[base + k] += add;
}

size_t scan_scratch_words(unsigned n) { return (n + kScanTile - 1) / kScanTile + 1; }

// In-place exclusive scan of a[0, n); the total goes to *total (device).
void scan_exclusive(unsigned* a, unsigned n, unsigned* scratch, unsigned* total, cudaStream_t st) {
  unsigned tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) {
    cudaMemsetAsync(total, 0, sizeof(unsigned), st);
    return;
  }
  k_scan_tiles<<<tiles, kScanThreads, 0, st>>>(a, n, scratch);
  count_launches(1);
  k_scan_sums<<<1, kScanThreads, 0, st>>>(scratch, tiles, total);
  count_launches(1);
  k_scan_add<<<tiles, 256, 0, st>>>(a, n, scratch);
  count_launches(1);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, kDevOk, code); }

// region vertex -> local id 2 + i; per-hypernode attributes of the region
__global__ void k_region_map(int32_t n, int32_t n_region, const int32_t* region,
                             const int32_t* side, const int32_t* node_w_h, int32_t* loc,
                             int32_t* node_gid, int32_t* node_w, int8_t* node_orig, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_region) return;
  int v = region[i];
  if (v < 0 || v >= n) { set_err(err, kDevBadInput); return; }
  int sd = side[v];
  if (sd != 0 && sd != 1) { set_err(err, kDevBadInput); return; }
  if (atomicExch(&loc[v], 2 + i) != -1) { set_err(err, kDevBadInput); return; }
  int c = node_w_h ? node_w_h[v] : 1;
  if (c <= 0) set_err(err, kDevBadInput);
  node_gid[2 + i] = v;
  node_w[2 + i] = c;
  node_orig[2 + i] = (int8_t)sd;
}

// contracted weights of s and t, and the total weight check
// verts (may be null): the vertices to scan (every vertex of side 0 or 1 must
// be among them); n is their count then, else all n vertices are scanned.
__global__ void k_st_weight(int32_t n, const int32_t* verts, const int32_t* loc,
                            const int32_t* side, const int32_t* node_w_h,
                            unsigned long long* wsum, int* err) {
  // wsum: [0] s, [1] t, [2] all of H, [3] nets (k_net_scan), [4] region
  __shared__ unsigned long long sh[5];
  if (threadIdx.x < 5) sh[threadIdx.x] = 0;
  __syncthreads();
  unsigned long long a0 = 0, a1 = 0, at = 0, ar = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int v = verts ? verts[i] : i;
    int c = node_w_h ? node_w_h[v] : 1;
    if (c <= 0) set_err(err, kDevBadInput);
    unsigned long long cc = (unsigned long long)(c > 0 ? c : 0);
    at += cc;
    if (loc[v] < 0) {
      int sd = side[v];
      if (sd == 0) a0 += cc;
      else if (sd == 1) a1 += cc;
    } else {
      ar += cc;
    }
  }
  if (a0) atomicAdd(&sh[0], a0);
  if (a1) atomicAdd(&sh[1], a1);
  if (at) atomicAdd(&sh[2], at);
  if (ar) atomicAdd(&sh[4], ar);
  __syncthreads();
  if (threadIdx.x < 5 && threadIdx.x != 3 && sh[threadIdx.x])
    atomicAdd(&wsum[threadIdx.x], sh[threadIdx.x]);
}

// pass 1, warp per net of H
// nets (may be null): the nets to scan, ascending (every net with a region
// pin must be among them); m is their count then.  Per-net outputs are
// indexed by the position in that list (by the net id without one).
__global__ void k_net_scan(int32_t n, int32_t m, const int32_t* nets, const uint32_t* net_off,
                           const int32_t* pins, const int32_t* net_w, const int32_t* side,
                           const int32_t* loc, unsigned* keep, unsigned* size, unsigned* has_s,
                           unsigned* has_t, int32_t* dist_tmp, int mark_dist,
                           unsigned long long* wnet, int* err) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long wacc = 0;
  for (unsigned i = gw; i < (unsigned)m; i += nw) {
    const unsigned e = nets ? (unsigned)nets[i] : i;
    const unsigned beg = net_off[e], end = net_off[e + 1];
    if (end < beg) { set_err(err, kDevBadInput); continue; }
    unsigned cnt = 0;
    bool hs = false, ht = false, s0 = false, s1 = false;
    for (unsigned j0 = beg; j0 < end; j0 += 32) {
      unsigned j = j0 + lane;
      bool reg = false, os = false, ot = false, a0 = false, a1 = false;
      if (j < end) {
        int v = pins[j];
        if (v < 0 || v >= n) {
          set_err(err, kDevBadInput);
        } else {
          int sd = side[v];
          a0 = sd == 0;
          a1 = sd == 1;
          reg = loc[v] >= 0;
          os = !reg && a0;
          ot = !reg && a1;
        }
      }
      cnt += __popc(__ballot_sync(FULLB, reg));
      hs |= __any_sync(FULLB, os);
      ht |= __any_sync(FULLB, ot);
      s0 |= __any_sync(FULLB, a0);
      s1 |= __any_sync(FULLB, a1);
    }
    const unsigned tot = cnt + hs + ht;
    const bool k = tot >= 2 && !(hs && ht);
    if (lane == 0) {
      int w = net_w[e];
      if (w <= 0) set_err(err, kDevBadInput);
      wacc += (unsigned long long)(w > 0 ? w : 0);
      keep[i] = k;
      size[i] = k ? tot : 0;
      has_s[i] = k && hs;
      has_t[i] = k && ht;
    }
    if (mark_dist && s0 && s1) {
      // region pins of a net with pins on both sides: distance 1
      for (unsigned j = beg + lane; j < end; j += 32) {
        int v = pins[j];
        if (v >= 0 && v < n) {
          int l = loc[v];
          if (l >= 0) dist_tmp[l - 2] = 1;   // indexed by region position
        }
      }
    }
  }
  if (lane == 0 && wacc) atomicAdd(wnet, wacc);
}

// pass 2, warp per net of H that is kept
__global__ void k_net_fill(int32_t m, const int32_t* nets, const uint32_t* net_off,
                           const int32_t* pins, const int32_t* net_w, const int32_t* loc,
                           const unsigned* keep,
                           const unsigned* net_pos, const unsigned* pin_pos,
                           const unsigned* s_pos, const unsigned* t_pos,
                           const unsigned* has_s_flag, const unsigned* has_t_flag,
                           const unsigned* totals, uint32_t* nnet_off, int32_t* npin,
                           int32_t* nnet_w, int32_t* nnet_gid, int2* inc) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned deg_s = totals[2];
  for (unsigned i = gw; i < (unsigned)m; i += nw) {
    if (!keep[i]) continue;
    const unsigned e = nets ? (unsigned)nets[i] : i;
    const unsigned beg = net_off[e], end = net_off[e + 1];
    const unsigned ep = net_pos[i];
    unsigned out = pin_pos[i];
    if (lane == 0) {
      nnet_off[ep] = out;
      nnet_w[ep] = net_w[e];
      nnet_gid[ep] = (int32_t)e;
    }
    for (unsigned j0 = beg; j0 < end; j0 += 32) {
      unsigned j = j0 + lane;
      int l = -1;
      if (j < end) l = loc[pins[j]];
      unsigned mask = __ballot_sync(FULLB, l >= 0);
      if (l >= 0) npin[out + __popc(mask & ((1u << lane) - 1u))] = l;
      out += __popc(mask);
    }
    if (lane == 0) {
      if (has_s_flag[i]) {
        npin[out] = 0;
        inc[s_pos[i]] = make_int2((int)ep, (int)out);
        out++;
      }
      if (has_t_flag[i]) {
        npin[out] = 1;
        inc[deg_s + t_pos[i]] = make_int2((int)ep, (int)out);
        out++;
      }
    }
  }
}

// incidence degrees of region hypernodes (s and t come from the scans)
__global__ void k_region_deg(const int32_t* npin, unsigned p, unsigned* deg) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < p; i += gridDim.x * blockDim.x) {
    int u = npin[i];
    if (u >= 2) atomicAdd(&deg[u], 1u);
  }
}

__global__ void k_set_st_deg(unsigned* deg, const unsigned* totals) {
  deg[0] = totals[2];
  deg[1] = totals[3];
}

// warp per kept net: scatter region incidences (order fixed by the sort below)
__global__ void k_region_inc(int32_t m_net, const uint32_t* nnet_off, const int32_t* npin,
                             const unsigned* node_off, unsigned* cursor, int2* inc) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m_net; e += nw) {
    for (unsigned p = nnet_off[e] + lane; p < nnet_off[e + 1]; p += 32) {
      int u = npin[p];
      if (u >= 2) inc[node_off[u] + atomicAdd(&cursor[u], 1u)] = make_int2((int)e, (int)p);
    }
  }
}

// warp per region hypernode: sort its incidences by pin slot (rank sort;
// slots are distinct).  Lists longer than 32 go through tmp.
__global__ void k_inc_sort(int32_t n_nodes, const unsigned* node_off, int2* inc, int2* tmp) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned u = 2 + gw; u < (unsigned)n_nodes; u += nw) {
    const unsigned beg = node_off[u], end = node_off[u + 1], d = end - beg;
    if (d <= 1) continue;
    if (d <= 32) {
      int2 mine = lane < d ? inc[beg + lane] : make_int2(0, 0x7fffffff);
      unsigned rank = 0;
      for (unsigned k = 0; k < d; k++) {
        int sk = __shfl_sync(FULLB, mine.y, k);
        rank += (sk < mine.y);
      }
      __syncwarp();
      if (lane < d) inc[beg + rank] = mine;
    } else {
      for (unsigned i = lane; i < d; i += 32) {
        int2 mine = inc[beg + i];
        unsigned rank = 0;
        for (unsigned k = 0; k < d; k++) rank += (inc[beg + k].y < mine.y);
        tmp[beg + rank] = mine;
      }
      __syncwarp();
      for (unsigned i = lane; i < d; i += 32) inc[beg + i] = tmp[beg + i];
    }
  }
}

// distance from the cut, initial values: 0 for s and t, 1 for region pins of
// nets with pins on both sides, -1 (not yet reached) otherwise; the engine's
// DIST states finish the breadth-first search on first use
__global__ void k_dist_seed(int32_t n_nodes, const int32_t* dist_tmp, int32_t* dist) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_nodes; u += gridDim.x * blockDim.x)
    dist[u] = u < 2 ? 0 : (dist_tmp[u - 2] == 1 ? 1 : -1);
}

// heavy bit: nodes with more arc groups than a lane handles go to a warp
__global__ void k_heavy_flags(const NetDev N) {
  const int nh = N.n_nodes, m = N.m_nets;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N.NL; x += gridDim.x * blockDim.x) {
    unsigned items;
    if (x < nh) {
      items = N.node_off[x + 1] - N.node_off[x];
    } else {
      const int e = x < nh + m ? x - nh : x - nh - m;
      items = 1 + N.net_off[e + 1] - N.net_off[e];
    }
    if (items > (unsigned)kLightItems) N.flags[x] |= kHeavy;
  }
}

// export copy: unreached vertices get the far distance
__global__ void k_dist_export(int32_t n_nodes, const int32_t* dist, int32_t* out) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n_nodes; u += gridDim.x * blockDim.x) {
    int d = dist[u];
    out[u] = (d < 0 || d > kDistFar) ? kDistFar : d;
  }
}

__global__ void k_dist_copy(int32_t n_region, const int32_t* dist_in, int32_t* dist, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    dist[0] = 0;
    dist[1] = 0;
  }
  if (i < n_region) {
    int d = dist_in[i];
    if (d < 0) set_err(err, kDevBadInput);
    dist[2 + i] = d > kDistFar ? kDistFar : d;
  }
}

__global__ void k_st_attrs(int32_t* node_gid, int32_t* node_w, int8_t* node_orig,
                           const unsigned long long* wsum, uint8_t* flags, int* err) {
  node_gid[0] = -1;
  node_gid[1] = -1;
  node_w[0] = (int32_t)wsum[0];
  node_w[1] = (int32_t)wsum[1];
  node_orig[0] = 0;
  node_orig[1] = 1;
  flags[0] = kSource;
  flags[1] = kSink;
  if (wsum[2] >= (1ull << 31)) set_err(err, kDevBadInput);
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// Second construction algorithm (Section 6, "Construction Algorithms"): the
// pairs (e, u) of every region vertex u and its nets e, sorted by net with
// the region order kept inside a net (a stable LSD radix sort), give the pin
// lists of the region's sub-hypergraph; s joins net e when fewer of e's pins
// of block 0 are in the region than e has in block 0, t likewise.  The work
// depends on the region's incidences only, not on the full pin lists of the
// nets that touch it.

// incidence count of every region vertex
__global__ void k_sb_deg(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                         unsigned* deg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
    const int v = region[i];
    deg[i] = vnet_off[v + 1] - vnet_off[v];
  }
}

// the pairs: key = net, value = local id 2 + i, grouped by region vertex
__global__ void k_sb_pairs(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                           const int32_t* vnet, const unsigned* pos, unsigned* key,
                           int32_t* val) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nr; i += gridDim.x * blockDim.x) {
    const int v = region[i];
    unsigned q = pos[i];
    for (unsigned t = vnet_off[v]; t < vnet_off[v + 1]; t++, q++) {
      key[q] = (unsigned)vnet[t];
      val[q] = 2 + i;
    }
  }
}

// Stable radix sort pass (8 bits at `shift`) over tiles of kRsTile items:
// per tile digit counts (digit-major), then a stable scatter by warp-level
// peer ranks and per-warp digit counts.
constexpr int kRsTile = 512;

__global__ void __launch_bounds__(kRsTile) k_rs_count(unsigned n, const unsigned* key, int shift,
                                                      unsigned T, unsigned* hist) {
  __shared__ unsigned cnt[256];
  for (int d = threadIdx.x; d < 256; d += blockDim.x) cnt[d] = 0;
  __syncthreads();
  const unsigned i = blockIdx.x * kRsTile + threadIdx.x;
  if (i < n) atomicAdd(&cnt[(key[i] >> shift) & 255u], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < 256; d += blockDim.x) hist[d * T + blockIdx.x] = cnt[d];
}

__global__ void __launch_bounds__(kRsTile) k_rs_scatter(unsigned n, const unsigned* key,
                                                        const int32_t* val, int shift, unsigned T,
                                                        const unsigned* hist, unsigned* key_out,
                                                        int32_t* val_out) {
  __shared__ unsigned wc[kRsTile / 32][256];
  const unsigned lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int j = threadIdx.x; j < (kRsTile / 32) * 256; j += blockDim.x) (&wc[0][0])[j] = 0;
  __syncthreads();
  const unsigned i = blockIdx.x * kRsTile + threadIdx.x;
  const bool in = i < n;
  const unsigned k = in ? key[i] : 0u;
  const unsigned d = in ? (k >> shift) & 255u : 256u;
  const unsigned peers = __match_any_sync(FULLB, d);
  const unsigned rank = __popc(peers & ((1u << lane) - 1u));
  if (in && rank == 0) wc[w][d] = __popc(peers);
  __syncthreads();
  for (int dd = threadIdx.x; dd < 256; dd += blockDim.x) {
    unsigned run = 0;
    for (int q = 0; q < kRsTile / 32; q++) {
      const unsigned c = wc[q][dd];
      wc[q][dd] = run;
      run += c;
    }
  }
  __syncthreads();
  if (in) {
    const unsigned o = hist[d * T + blockIdx.x] + wc[w][d] + rank;
    key_out[o] = k;
    val_out[o] = val[i];
  }
}

// first pair of every net (run head)
__global__ void k_sb_heads(unsigned n, const unsigned* key, unsigned* head) {
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    head[j] = (j == 0 || key[j] != key[j - 1]) ? 1u : 0u;
}

// run_start[R] = the pair count (R = the number of runs, at *R)
__global__ void k_sb_end(unsigned* run_start, const unsigned* R, unsigned n) { run_start[*R] = n; }

__global__ void k_sb_runs(unsigned n, const unsigned* key, const unsigned* head,
                          const unsigned* rid, unsigned* run_start, int32_t* run_net) {
  for (unsigned j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    if (head[j]) {
      run_start[rid[j]] = j;
      run_net[rid[j]] = (int32_t)key[j];
    }
}

// per net of the region: region pins by side, pins of the two blocks in H
// (cnt[noff[e] + rank of the block in the net's mask]), s / t membership,
// kept size (the first algorithm's rules)
__global__ void k_sb_eval(unsigned R, const unsigned* run_start, const int32_t* run_net,
                          const int32_t* val, const int32_t* region, const int32_t* side,
                          const int32_t* net_w, const unsigned long long* mask,
                          const unsigned* noff, const unsigned* cnt, int32_t b0, int32_t b1,
                          unsigned* keep, unsigned* size, unsigned* has_s, unsigned* has_t,
                          unsigned long long* wnet) {
  unsigned long long wacc = 0;
  for (unsigned r = blockIdx.x * blockDim.x + threadIdx.x; r < R; r += gridDim.x * blockDim.x) {
    const int e = run_net[r];
    unsigned in0 = 0, in1 = 0;
    for (unsigned j = run_start[r]; j < run_start[r + 1]; j++) {
      const int sd = side[region[val[j] - 2]];
      in0 += sd == 0;
      in1 += sd == 1;
    }
    const unsigned long long mk = mask[e];
    const unsigned tot0 = (mk >> b0) & 1ull
                              ? cnt[noff[e] + __popcll(mk & ((1ull << b0) - 1ull))] : 0u;
    const unsigned tot1 = (mk >> b1) & 1ull
                              ? cnt[noff[e] + __popcll(mk & ((1ull << b1) - 1ull))] : 0u;
    const bool hs = in0 < tot0, ht = in1 < tot1;
    const unsigned tot = in0 + in1 + hs + ht;
    const bool k = tot >= 2 && !(hs && ht);
    keep[r] = k;
    size[r] = k ? tot : 0;
    has_s[r] = k && hs;
    has_t[r] = k && ht;
    wacc += (unsigned long long)net_w[e];
  }
  if (wacc) atomicAdd(wnet, wacc);
}

// the kept nets' pin lists (region pins in region order, then s, then t),
// weights, ids in H and s / t incidences, a warp per net
__global__ void k_sb_fill(unsigned R, const unsigned* run_start, const int32_t* run_net,
                          const int32_t* val, const int32_t* side, const int32_t* region,
                          const int32_t* net_w, const unsigned* keep, const unsigned* net_pos,
                          const unsigned* pin_pos, const unsigned* s_pos, const unsigned* t_pos,
                          const unsigned* has_s_flag, const unsigned* has_t_flag,
                          const unsigned* totals, uint32_t* nnet_off, int32_t* npin,
                          int32_t* nnet_w, int32_t* nnet_gid, int2* inc) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  const unsigned deg_s = totals[2];
  for (unsigned r = gw; r < R; r += nw) {
    if (!keep[r]) continue;
    const unsigned beg = run_start[r], end = run_start[r + 1];
    const unsigned ep = net_pos[r];
    unsigned out = pin_pos[r];
    const int e = run_net[r];
    if (lane == 0) {
      nnet_off[ep] = out;
      nnet_w[ep] = net_w[e];
      nnet_gid[ep] = e;
    }
    for (unsigned j0 = beg; j0 < end; j0 += 32) {
      const unsigned j = j0 + lane;
      int l = -1;
      if (j < end) {
        l = val[j];
        const int sd = side[region[l - 2]];
        if (sd != 0 && sd != 1) l = -1;
      }
      const unsigned mk = __ballot_sync(FULLB, l >= 0);
      if (l >= 0) npin[out + __popc(mk & ((1u << lane) - 1u))] = l;
      out += __popc(mk);
    }
    if (lane == 0) {
      if (has_s_flag[r]) {
        npin[out] = 0;
        inc[s_pos[r]] = make_int2((int)ep, (int)out);
        out++;
      }
      if (has_t_flag[r]) {
        npin[out] = 1;
        inc[deg_s + t_pos[r]] = make_int2((int)ep, (int)out);
        out++;
      }
    }
  }
}

static inline unsigned blocks_for(unsigned long long work, unsigned per_block, unsigned cap) {
  unsigned long long b = (work + per_block - 1) / per_block;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

void launch_region_map(int32_t n, int32_t n_region, const int32_t* region, const int32_t* side,
                       const int32_t* node_w_h, int32_t* loc, int32_t* node_gid, int32_t* node_w,
                       int8_t* node_orig, int* err, cudaStream_t st) {
  if (n_region > 0) {
    k_region_map<<<(n_region + 255) / 256, 256, 0, st>>>(n, n_region, region, side, node_w_h, loc,
                                                        node_gid, node_w, node_orig, err);
    count_launches(1);
  }
}

void launch_st_weight(int32_t n, const int32_t* verts, const int32_t* loc, const int32_t* side,
                      const int32_t* node_w_h, unsigned long long* wsum, int* err, int sms,
                      cudaStream_t st) {
  k_st_weight<<<blocks_for(n, 256, sms * 8), 256, 0, st>>>(n, verts, loc, side, node_w_h, wsum,
                                                            err);
  count_launches(1);
}

void launch_net_scan(int32_t n, int32_t m, const int32_t* nets, const uint32_t* net_off,
                     const int32_t* pins, const int32_t* net_w, const int32_t* side,
                     const int32_t* loc, unsigned* keep, unsigned* size, unsigned* has_s,
                     unsigned* has_t, int32_t* dist_tmp, int mark_dist, unsigned long long* wnet,
                     int* err, int sms, cudaStream_t st) {
  if (m > 0) {
    k_net_scan<<<blocks_for((unsigned long long)m * 32, 256, sms * 16), 256, 0, st>>>(
        n, m, nets, net_off, pins, net_w, side, loc, keep, size, has_s, has_t, dist_tmp,
        mark_dist, wnet, err);
    count_launches(1);
  }
}

void launch_net_fill(int32_t m, const int32_t* nets, const uint32_t* net_off,
                     const int32_t* pins, const int32_t* net_w, const int32_t* loc,
                     const unsigned* keep,
                     const unsigned* net_pos, const unsigned* pin_pos, const unsigned* s_pos,
                     const unsigned* t_pos, const unsigned* has_s, const unsigned* has_t,
                     const unsigned* totals, uint32_t* nnet_off, int32_t* npin, int32_t* nnet_w,
                     int32_t* nnet_gid, int2* inc, int sms, cudaStream_t st) {
  if (m > 0) {
    k_net_fill<<<blocks_for((unsigned long long)m * 32, 256, sms * 16), 256, 0, st>>>(
        m, nets, net_off, pins, net_w, loc, keep, net_pos, pin_pos, s_pos, t_pos, has_s, has_t,
        totals, nnet_off, npin, nnet_w, nnet_gid, inc);
    count_launches(1);
  }
}

void launch_incidence(int32_t n_nodes, int32_t m_net, unsigned p, const uint32_t* nnet_off,
                      const int32_t* npin, unsigned* deg_then_off, unsigned* cursor,
                      const unsigned* totals, int2* inc, int2* tmp, unsigned* scan_scratch,
                      unsigned* scan_total, int sms, cudaStream_t st) {
  cudaMemsetAsync(deg_then_off, 0, sizeof(unsigned) * (n_nodes + 1), st);
  if (p > 0) {
    k_region_deg<<<blocks_for(p, 256, sms * 8), 256, 0, st>>>(npin, p, deg_then_off);
    count_launches(1);
  }
  k_set_st_deg<<<1, 1, 0, st>>>(deg_then_off, totals);
  count_launches(1);
  scan_exclusive(deg_then_off, n_nodes + 1, scan_scratch, scan_total, st);
  cudaMemsetAsync(cursor, 0, sizeof(unsigned) * n_nodes, st);
  if (m_net > 0) {
    k_region_inc<<<blocks_for((unsigned long long)m_net * 32, 256, sms * 16), 256, 0, st>>>(
        m_net, nnet_off, npin, deg_then_off, cursor, inc);
    count_launches(1);
  }
  if (n_nodes > 2) {
    k_inc_sort<<<blocks_for((unsigned long long)n_nodes * 32, 256, sms * 16), 256, 0, st>>>(
        n_nodes, deg_then_off, inc, tmp);
    count_launches(1);
  }
}

void launch_dist_seed(int32_t n_nodes, const int32_t* dist_tmp, int32_t* dist, int sms,
                      cudaStream_t st) {
  k_dist_seed<<<blocks_for(n_nodes, 256, sms * 8), 256, 0, st>>>(n_nodes, dist_tmp, dist);
  count_launches(1);
}

void launch_heavy_flags(const NetDev& N, int sms, cudaStream_t st) {
  k_heavy_flags<<<blocks_for(N.NL, 256, sms * 8), 256, 0, st>>>(N);
  count_launches(1);
}

void launch_dist_export(int32_t n_nodes, const int32_t* dist, int32_t* out, int sms,
                        cudaStream_t st) {
  k_dist_export<<<blocks_for(n_nodes, 256, sms * 8), 256, 0, st>>>(n_nodes, dist, out);
  count_launches(1);
}

void launch_dist_copy(int32_t n_region, const int32_t* dist_in, int32_t* dist, int* err,
                      cudaStream_t st) {
  k_dist_copy<<<(n_region + 2 + 255) / 256, 256, 0, st>>>(n_region, dist_in, dist, err);
  count_launches(1);
}

void launch_st_attrs(int32_t* node_gid, int32_t* node_w, int8_t* node_orig,
                     const unsigned long long* wsum, uint8_t* flags, int* err, cudaStream_t st) {
  k_st_attrs<<<1, 1, 0, st>>>(node_gid, node_w, node_orig, wsum, flags, err);
  count_launches(1);
}

// ---------------------------------------------------------------------------
// Identical net removal (Section 6, "Identical Net Removal").  Nets of the
// built flow hypergraph are grouped by a tag derived from the paper's
// fingerprint sum of v^2, the size and an order-independent 64-bit mix of
// the pins; within a group the smallest net id is found with atomicMin in an
// open-addressing table, and a net merges into it when the two pin sets are
// equal (compared pin by pin).  Nets with identical sets always share a tag,
// so every net merges into the smallest-id net with its set (two different
// sets with one tag would only leave a merge undone).  Kept nets stay in
// ascending order; the representative carries the summed weight.

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64's output function (Steele, Lea and Flood, 2014)
  z ^= z >> 30;
  z *= 0xbf58476d1ce4e5b9ull;
  z ^= z >> 27;
  z *= 0x94d049bb133111ebull;
  z ^= z >> 31;
  return z;
}

// warp per net: the group tag (never 0)
__global__ void k_net_tag(int32_t m, const uint32_t* off, const int32_t* pin,
                          unsigned long long* tag) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    unsigned long long f = 0, h = 0;
    for (unsigned p = off[e] + lane; p < off[e + 1]; p += 32) {
      const unsigned long long v = (unsigned)pin[p];
      f += v * v;
      h += mix64(v + 0x9e3779b97f4a7c15ull);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      f += __shfl_xor_sync(FULLB, f, o);
      h += __shfl_xor_sync(FULLB, h, o);
    }
    if (lane == 0) {
      const unsigned long long size = off[e + 1] - off[e];
      tag[e] = mix64(f ^ mix64(h ^ (size << 40))) | 1ull;
    }
  }
}

// smallest net id per tag (open addressing, linear probing; the table has
// at least twice as many slots as nets, so a probe always ends)
__global__ void k_tag_insert(int32_t m, const unsigned long long* tag, unsigned long long* tab_tag,
                             int32_t* tab_min, unsigned mask, int* err) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    const unsigned long long t = tag[e];
    unsigned slot = (unsigned)(t >> 20) & mask;
    for (unsigned probe = 0;; probe++) {
      if (probe > mask) {
        atomicExch(err, 1);
        break;
      }
      const unsigned long long old = atomicCAS(&tab_tag[slot], 0ull, t);
      if (old == 0ull || old == t) {
        atomicMin(&tab_min[slot], e);
        break;
      }
      slot = (slot + 1) & mask;
    }
  }
}

// warp per net: its representative (the group's smallest id when the pin
// sets are equal, else itself)
__global__ void k_net_rep(int32_t m, const uint32_t* off, const int32_t* pin,
                          const unsigned long long* tag, const unsigned long long* tab_tag,
                          const int32_t* tab_min, unsigned mask, int32_t* rep) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    const unsigned long long t = tag[e];
    unsigned slot = (unsigned)(t >> 20) & mask;
    for (unsigned probe = 0; probe <= mask && tab_tag[slot] != t; probe++) slot = (slot + 1) & mask;
    const int r = tab_tag[slot] == t ? tab_min[slot] : (int)e;
    bool same = r != (int)e;
    if (same) {
      // sizes are equal (part of the tag); every pin of e must occur in r
      const unsigned b = off[e], size = off[e + 1] - b, rb = off[r];
      bool all = true;
      for (unsigned i = lane; i < size; i += 32) {
        const int v = pin[b + i];
        bool found = false;
        for (unsigned j = 0; j < size && !found; j++) found = pin[rb + j] == v;
        all = all && found;
      }
      same = __all_sync(FULLB, all);
    }
    if (lane == 0) rep[e] = same ? r : (int)e;
  }
}

// weights to representatives; kept-net flags and sizes; s / t membership
__global__ void k_net_merge(int32_t m, const uint32_t* off, const int32_t* pin,
                            const int32_t* net_w, const int32_t* rep, unsigned long long* wacc,
                            unsigned* keep, unsigned* size, unsigned* has_s, unsigned* has_t) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    atomicAdd(&wacc[rep[e]], (unsigned long long)net_w[e]);
    const bool k = rep[e] == e;
    const unsigned sz = off[e + 1] - off[e];
    const int last = pin[off[e + 1] - 1];   // s, then t, come after the region pins
    keep[e] = k ? 1u : 0u;
    size[e] = k ? sz : 0u;
    has_s[e] = k && last == 0 ? 1u : 0u;
    has_t[e] = k && last == 1 ? 1u : 0u;
  }
}

// warp per kept net: copy to its compacted place
__global__ void k_net_compact(int32_t m, const uint32_t* off, const int32_t* pin,
                              const int32_t* gid, const unsigned* keep, const unsigned* new_e,
                              const unsigned* new_p, const unsigned long long* wacc,
                              uint32_t* o_off, int32_t* o_pin, int32_t* o_w, int32_t* o_gid) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    if (!keep[e]) continue;
    const unsigned ne = new_e[e], np = new_p[e], b = off[e], size = off[e + 1] - b;
    for (unsigned i = lane; i < size; i += 32) o_pin[np + i] = pin[b + i];
    if (lane == 0) {
      o_off[ne] = np;
      o_w[ne] = (int32_t)wacc[e];
      o_gid[ne] = gid[e];
    }
  }
}

// s / t incidences of the compacted nets, in ascending net order
__global__ void k_st_inc(int32_t m, const uint32_t* off, const unsigned* keep,
                         const unsigned* new_e, const unsigned* has_s, const unsigned* has_t,
                         const unsigned* pos_s, const unsigned* pos_t, const unsigned* node_off,
                         const uint32_t* n_off, int2* inc) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < m; e += gridDim.x * blockDim.x) {
    if (!keep[e]) continue;
    const int ne = (int)new_e[e];
    const int slot = (int)n_off[ne + 1] - 1;
    if (has_s[e]) inc[node_off[0] + pos_s[e]] = make_int2(ne, slot);
    if (has_t[e]) inc[node_off[1] + pos_t[e]] = make_int2(ne, slot);
  }
}

__global__ void k_dedup_totals(unsigned m_new, unsigned p_new, const unsigned* has_s_tot,
                               const unsigned* has_t_tot, uint32_t* n_off, unsigned* totals) {
  n_off[m_new] = p_new;
  totals[0] = m_new;
  totals[1] = p_new;
  totals[2] = *has_s_tot;
  totals[3] = *has_t_tot;
}

void launch_net_tags(int32_t m, const uint32_t* off, const int32_t* pin, unsigned long long* tag,
                     unsigned long long* tab_tag, int32_t* tab_min, unsigned mask, int32_t* rep,
                     int* err, int sms, cudaStream_t st) {
  if (m <= 0) return;
  const unsigned wb = blocks_for((unsigned long long)m * 32, 256, sms * 16);
  k_net_tag<<<wb, 256, 0, st>>>(m, off, pin, tag);
  k_tag_insert<<<blocks_for(m, 256, sms * 8), 256, 0, st>>>(m, tag, tab_tag, tab_min, mask, err);
  k_net_rep<<<wb, 256, 0, st>>>(m, off, pin, tag, tab_tag, tab_min, mask, rep);
  count_launches(3);
}

void launch_net_merge(int32_t m, const uint32_t* off, const int32_t* pin, const int32_t* net_w,
                      const int32_t* rep, unsigned long long* wacc, unsigned* keep,
                      unsigned* size, unsigned* has_s, unsigned* has_t, int sms,
                      cudaStream_t st) {
  if (m <= 0) return;
  k_net_merge<<<blocks_for(m, 256, sms * 8), 256, 0, st>>>(m, off, pin, net_w, rep, wacc, keep,
                                                          size, has_s, has_t);
  count_launches(1);
}

void launch_net_compact(int32_t m, const uint32_t* off, const int32_t* pin, const int32_t* gid,
                        const unsigned* keep, const unsigned* new_e, const unsigned* new_p,
                        const unsigned long long* wacc, uint32_t* o_off, int32_t* o_pin,
                        int32_t* o_w, int32_t* o_gid, int sms, cudaStream_t st) {
  if (m <= 0) return;
  k_net_compact<<<blocks_for((unsigned long long)m * 32, 256, sms * 16), 256, 0, st>>>(
      m, off, pin, gid, keep, new_e, new_p, wacc, o_off, o_pin, o_w, o_gid);
  count_launches(1);
}

void launch_dedup_totals(unsigned m_new, unsigned p_new, const unsigned* has_s_tot,
                         const unsigned* has_t_tot, uint32_t* n_off, unsigned* totals,
                         cudaStream_t st) {
  k_dedup_totals<<<1, 1, 0, st>>>(m_new, p_new, has_s_tot, has_t_tot, n_off, totals);
  count_launches(1);
}

void launch_st_inc(int32_t m, const uint32_t* off, const unsigned* keep, const unsigned* new_e,
                   const unsigned* has_s, const unsigned* has_t, const unsigned* pos_s,
                   const unsigned* pos_t, const unsigned* node_off, const uint32_t* n_off,
                   int2* inc, int sms, cudaStream_t st) {
  if (m <= 0) return;
  k_st_inc<<<blocks_for(m, 256, sms * 8), 256, 0, st>>>(m, off, keep, new_e, has_s, has_t, pos_s,
                                                       pos_t, node_off, n_off, inc);
  count_launches(1);
}

// Second construction algorithm, pass 1: the region's (net, vertex) pairs
// sorted by net; returns the number of nets touching the region (*R) and
// fills run_start[R + 1] / run_net[R] (buffers of at least the pair count;
// key/val and key2/val2 of the pair count).  Synchronises.
cudaError_t sort_build_count(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                             unsigned* deg, unsigned* scr, unsigned* tot, unsigned* n_pairs,
                             int sms, cudaStream_t st) {
  *n_pairs = 0;
  if (nr <= 0) return cudaSuccess;
  k_sb_deg<<<blocks_for(nr, 256, sms * 8), 256, 0, st>>>(nr, region, vnet_off, deg);
  count_launches(1);
  scan_exclusive(deg, (unsigned)nr, scr, tot, st);
  cudaError_t ce = cudaMemcpyAsync(n_pairs, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  return ce;
}

cudaError_t sort_build_runs(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                            const int32_t* vnet, int32_t m, unsigned P2, const unsigned* pos,
                            unsigned* scr, unsigned* tot, unsigned* key, int32_t* val,
                            unsigned* key2, int32_t* val2, unsigned* hist, unsigned* head,
                            unsigned* rid, unsigned* run_start, int32_t* run_net, unsigned* R,
                            int sms, cudaStream_t st) {
  *R = 0;
  cudaError_t ce = cudaSuccess;
  if (P2 == 0) return cudaSuccess;
  k_sb_pairs<<<blocks_for(nr, 256, sms * 8), 256, 0, st>>>(nr, region, vnet_off, vnet, pos, key,
                                                           val);
  count_launches(1);
  const unsigned T = (P2 + kRsTile - 1) / kRsTile;
  int bits = 1;
  while (bits < 31 && (1u << bits) < (unsigned)m) bits++;
  unsigned *ka = key, *kb = key2;
  int32_t *va = val, *vb = val2;
  for (int shift = 0; shift < bits; shift += 8) {
    k_rs_count<<<T, kRsTile, 0, st>>>(P2, ka, shift, T, hist);
    scan_exclusive(hist, 256 * T, scr, tot, st);
    k_rs_scatter<<<T, kRsTile, 0, st>>>(P2, ka, va, shift, T, hist, kb, vb);
    count_launches(2);
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  // the sorted pairs end in key / val
  if (ka != key) {
    ce = cudaMemcpyAsync(key, ka, sizeof(unsigned) * P2, cudaMemcpyDeviceToDevice, st);
    if (ce == cudaSuccess)
      ce = cudaMemcpyAsync(val, va, sizeof(int32_t) * P2, cudaMemcpyDeviceToDevice, st);
    if (ce != cudaSuccess) return ce;
  }
  // runs of equal nets
  k_sb_heads<<<blocks_for(P2, 256, sms * 8), 256, 0, st>>>(P2, key, head);
  count_launches(1);
  ce = cudaMemcpyAsync(rid, head, sizeof(unsigned) * P2, cudaMemcpyDeviceToDevice, st);
  if (ce != cudaSuccess) return ce;
  scan_exclusive(rid, P2, scr, tot, st);
  k_sb_runs<<<blocks_for(P2, 256, sms * 8), 256, 0, st>>>(P2, key, head, rid, run_start, run_net);
  k_sb_end<<<1, 1, 0, st>>>(run_start, tot, P2);
  count_launches(2);
  unsigned r = 0;
  ce = cudaMemcpyAsync(&r, tot, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
  *R = r;
  return ce;
}

void launch_sb_eval(unsigned R, const unsigned* run_start, const int32_t* run_net,
                    const int32_t* val, const int32_t* region, const int32_t* side,
                    const int32_t* net_w, const unsigned long long* mask, const unsigned* noff,
                    const unsigned* cnt, int32_t b0, int32_t b1, unsigned* keep, unsigned* size,
                    unsigned* has_s, unsigned* has_t, unsigned long long* wnet, int sms,
                    cudaStream_t st) {
  if (R == 0) return;
  k_sb_eval<<<blocks_for(R, 256, sms * 8), 256, 0, st>>>(R, run_start, run_net, val, region, side,
                                                         net_w, mask, noff, cnt, b0, b1, keep,
                                                         size, has_s, has_t, wnet);
  count_launches(1);
}

void launch_sb_fill(unsigned R, const unsigned* run_start, const int32_t* run_net,
                    const int32_t* val, const int32_t* side, const int32_t* region,
                    const int32_t* net_w, const unsigned* keep, const unsigned* net_pos,
                    const unsigned* pin_pos, const unsigned* s_pos, const unsigned* t_pos,
                    const unsigned* has_s, const unsigned* has_t, const unsigned* totals,
                    uint32_t* nnet_off, int32_t* npin, int32_t* nnet_w, int32_t* nnet_gid,
                    int2* inc, int sms, cudaStream_t st) {
  if (R == 0) return;
  k_sb_fill<<<blocks_for((unsigned long long)R * 32, 256, sms * 16), 256, 0, st>>>(
      R, run_start, run_net, val, side, region, net_w, keep, net_pos, pin_pos, s_pos, t_pos,
      has_s, has_t, totals, nnet_off, npin, nnet_w, nnet_gid, inc);
  count_launches(1);
}

}  // namespace hfp

