// Shared device/host definitions of the hfp CUDA library (sm_103a).
//
// Flow hypergraph layout in HBM (one hfp_net):
//   hypernodes h in [0, n_nodes): 0 = s, 1 = t, 2 + i = region[i]
//   Lawler ids:  hypernode h -> h;  in-node of net e -> n_nodes + e;
//                out-node of net e -> n_nodes + m_nets + e     (Section 2)
//   net_off[m+1], pin[p]            net -> pins (pin slots)
//   node_off[n+1], inc[p] (int2)    hypernode -> (net, pin slot)
//   f_in[p]  flow on (u, e_in) of pin slot p   (capped at w(e), Section 8.3)
//   f_out[p] flow on (e_out, u) of pin slot p
//   f_b[m]   flow on the bridge (e_in, e_out)
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace hfp {

constexpr int kWarp = 32;

// per Lawler node flag bits (flags[])
constexpr uint8_t kSource = 1;
constexpr uint8_t kSink = 2;
constexpr uint8_t kHeavy = 4;      // more than kLightItems arc groups: a warp per node
constexpr uint8_t kTerminal = kSource | kSink;

// A node is light when its arc scan has at most kLightItems steps (a
// hypernode's incidences; a net node's bridge plus pins); light nodes are
// handled one per lane, heavy ones one per warp.
constexpr int kLightItems = 16;

// device error codes (ctl->err); host maps them to hfp_status
constexpr int kDevOk = 0;
constexpr int kDevTimeout = 1;     // a bounded spin gave up
constexpr int kDevIterLimit = 2;   // round / relabel budget exhausted
constexpr int kDevBadInput = 3;    // bounds or duplicate check failed

struct NetDev {
  int32_t n_nodes, m_nets, NL;  // hypernodes, nets, Lawler nodes
  int64_t p_pins;
  const uint32_t* net_off;
  const int32_t* pin;
  const int32_t* net_w;
  const uint32_t* node_off;
  const int2* inc;              // (net, pin slot), sorted by slot per node
  const int32_t* node_w;
  int32_t* node_dist;           // distance from the original cut (-1: not reached yet)
  const int8_t* node_orig;      // original side (0/1) per hypernode
  const int32_t* node_gid;      // id in H (-1 for s, t)
  int32_t* f_in;
  int32_t* f_out;
  int32_t* f_b;
  int32_t* lab0;                // labels, double buffered by round parity
  int32_t* lab1;
  long long* excess;
  long long* delta;
  long long* delta1;            // second delta buffer of one-phase rounds (may be null)
  uint32_t* stamp;
  uint8_t* flags;
  uint8_t* needrl;
  uint8_t* insr;                // forward residual reachability (S_r)
  int32_t* list[4];             // frontier, next, relabeled, BFS lists (NL each)
  unsigned long long* trace;    // per-phase trace (4 words per phase), may be null
  unsigned int trace_cap;       // phases the trace can hold
  unsigned int gq_cap;          // entries of gq
  unsigned long long* gq;       // work queue of the asynchronous global relabel (may be null)
  uint8_t* net_done;            // per net: every pin is a terminal (batched piercing scans;
                                // may be null)
  uint32_t* blk;                // per node: ParPR-Block tag of the running round (may be null)
};

struct Ctl {
  unsigned long long flow;      // flow value: excess that reached the sinks
  int err;                      // kDev* code, first error wins
  int err_where;
  unsigned long long rounds, global_relabels, gr_levels;
  unsigned long long work_since_gr;  // arcs scanned since the last global relabel
  unsigned long long items_hyper;    // hypernode incidences scanned (all phases)
  unsigned long long items_net;      // net pins scanned (all phases)
  unsigned long long node_visits;    // frontier / list entries processed
  unsigned long long pushes;
  unsigned long long stall_rounds;
  long long wS, wT;             // c(S_r), c(T_r): hypernode weights
  unsigned long long best_key;  // piercing candidate selection
  int best_node;
  int pad;
  // tracing: device time between grid barriers, by engine state (globaltimer)
  unsigned long long state_ns[10];
  unsigned long long state_cnt[10];
  unsigned long long trace_len;   // entries written to the round trace
  unsigned long long gq_items;    // asynchronous global relabels: queue entries expanded
  unsigned long long gq_overs;    // ... and relabels redone level by level (queue full)
};

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ void st_release(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Release reduction: every write this thread has made or observed (including,
// through a preceding __syncthreads, those of its CTA) is visible before the
// addition is.
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread-block cluster helpers.  `addr` is a shared::cluster address (mapa).
__device__ __forceinline__ unsigned dsmem_addr(const void* smem, unsigned rank) {
  const unsigned local = (unsigned)__cvta_generic_to_shared(smem);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(local), "r"(rank));
  return r;
}

__device__ __forceinline__ void dsmem_red_release_add(unsigned addr, unsigned v) {
  asm volatile("red.release.cluster.shared::cluster.add.u32 [%0], %1;" ::"r"(addr), "r"(v)
               : "memory");
}

__device__ __forceinline__ unsigned dsmem_ld_acquire(unsigned addr) {
  unsigned v;
  asm volatile("ld.acquire.cluster.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(addr) : "memory");
  return v;
}

// Hardware barrier of all threads of the cluster (every thread must call it).
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Count-up barrier arithmetic that survives wrap-around of the counter.
__device__ __forceinline__ bool count_reached(unsigned v, unsigned target) {
  return (int)(v - target) >= 0;
}

__device__ __forceinline__ int ld_volatile_int(const int* p) {
  return *(const volatile int*)p;
}

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

// Warp-aggregated append of `want` lanes to list[] at counter *cnt.
// All 32 lanes of the warp must call it together.
__device__ __forceinline__ void warp_append(bool want, int32_t value, int32_t* list,
                                            unsigned int* cnt) {
  unsigned mask = __ballot_sync(0xffffffffu, want);
  if (!mask) return;
  unsigned lane = lane_id();
  unsigned base = 0;
  int leader = __ffs(mask) - 1;
  if ((int)lane == leader) base = atomicAdd(cnt, (unsigned)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (want) list[base + __popc(mask & ((1u << lane) - 1u))] = value;
}

__device__ __forceinline__ long long warp_incl_scan(long long v) {
  unsigned lane = lane_id();
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long t = __shfl_up_sync(0xffffffffu, v, o);
    if ((int)lane >= o) v += t;
  }
  return v;
}

__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_min(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// MurmurHash3's 32-bit finaliser (Appleby), a bijection on 32-bit words:
// the third piercing key.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

}  // namespace hfp
