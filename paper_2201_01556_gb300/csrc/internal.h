// Host-side internals shared by the C ABI translation units (api.cu,
// kway.cu): context and network objects, error reporting, stream-ordered
// device buffers.
#pragma once
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "hfp.h"
#include "kernels.cuh"

#define HFP_API extern "C" __attribute__((visibility("default")))

namespace hfp {

// Records a message for hfp_last_error and returns s.
hfp_status fail(hfp_status s, const char* fmt, ...);
void set_last_error(const char* msg);

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return ::hfp::fail(e_ == cudaErrorMemoryAllocation ? HFP_ERR_OOM : HFP_ERR_CUDA,    \
                         "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                       \
  } while (0)

// Stream-ordered device allocation owned by a scope.
struct DevBuf {
  void* p = nullptr;
  cudaStream_t st = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
  cudaError_t alloc(size_t bytes, cudaStream_t s) {
    st = s;
    return cudaMallocAsync(&p, bytes ? bytes : 16, s);
  }
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Engine knobs of a batched launch (the context's, or an autotuner's pick).
struct BatchTune {
  Params P;
  uint32_t gr_work_x100;
};

}  // namespace hfp

struct hfp_ctx {
  std::atomic<int> refs{1};        // the caller's handle + one per live network
  int device = 0;
  cudaStream_t stream = nullptr;
  int sms = 0;
  int coop_grid = 0;
  int threads = hfp::kEngineThreads;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // engine launch timing
  hfp::Ctl* pinned_ctl = nullptr;  // host mirror of Ctl
  void* pinned_small = nullptr;    // 4 KB staging
  hfp::Params params{};
  uint32_t gr_work_x100 = 200;
  uint32_t batch_cluster = 1;      // hfp_tuning.batch_cluster
  uint32_t batch_big_ctas = 0;     // hfp_tuning.batch_big_ctas
  uint32_t batch_big_groups = 0;   // hfp_tuning.batch_big_groups
  uint32_t identical_nets = 0;     // hfp_tuning.identical_nets
  uint32_t batch_fused_rounds = 1; // hfp_tuning.batch_fused_rounds
  uint32_t batch_async_gr = 0;     // hfp_tuning.batch_async_gr
  uint32_t construction = 1;       // hfp_tuning.construction
  uint32_t batch_gr_work_x100 = 100;       // hfp_tuning.batch_gr_work_x100
  uint32_t batch_stall_rounds_pierce = 30; // hfp_tuning.batch_stall_rounds_pierce
  uint32_t prep_streams = 8;       // hfp_tuning.prep_streams
  int32_t last_groups = 0, last_group_ctas = 0, last_cluster = 0;   // last batched launch
  bool owns_stream = false;        // a helper context's stream (destroyed with it)
  // group time per engine state of the batched launches since the last reset
  uint64_t batch_ns[hfp::kStateSlots] = {};
  uint64_t batch_cnt[hfp::kStateSlots] = {};
  uint64_t batch_lin[hfp::kStateSlots] = {};
  uint64_t batch_hin[hfp::kStateSlots] = {};
};

struct hfp_net {
  hfp_ctx* ctx = nullptr;
  hfp::NetDev d{};
  hfp::EngineCtl* E = nullptr;
  void* arena = nullptr;
  int32_t* net_gid = nullptr;
  int32_t* dev_nodes = nullptr;    // staging for pierced node ids
  int32_t dev_nodes_cap = 0;
  int32_t n_region = 0;
  int64_t total_w = 0;
  bool flow_started = false;
  bool labels_exact = false;
  bool sr_valid = false;
  bool dist_ready = false;
  // a source pierced without augmenting path whose arcs were left unsaturated
  // (saturated before the next sink-side piercing), and the seed of the next
  // incremental source-side search (-1: a full search is needed)
  int32_t pending_source = -1;
  int32_t sr_seed = -1;
  // a sink was pierced without augmenting path: T_r was grown by a search from
  // it, so the labels are no longer exact distances and the next flow
  // computation starts with a global relabel
  bool gr_pending = false;
  bool pierced = false;            // flows from now on are incremental
  void* trace_buf = nullptr;
  void* gq_buf = nullptr;          // work queue of queue-driven global relabels
  void* delta1_buf = nullptr;      // second delta buffer of one-phase rounds
  void* net_done_buf = nullptr;    // nets the batched piercing scans skip
  void* blk_buf = nullptr;         // ParPR-Block tags
  uint64_t launches = 0;
  uint64_t engine_ns = 0;
};

// Device-resident hypergraph of the k-way calls (kway.cu, sched.cu).
struct hfp_hgraph {
  hfp_ctx* ctx = nullptr;
  int32_t n = 0, m = 0;
  int64_t p = 0;
  int64_t total_w = 0;
  void* arena = nullptr;
  uint32_t* net_off = nullptr;
  int32_t* pins = nullptr;
  int32_t* net_w = nullptr;
  int32_t* node_w = nullptr;
  uint32_t* vnet_off = nullptr;   // vertex -> nets incidence (ascending net ids)
  int32_t* vnet = nullptr;
  int32_t tuned_group = 0;        // CTAs per FlowCutter problem picked by hfp_autotune_round
  bool tuned_engine = false;      // engine knobs picked by hfp_autotune_round_engine
  hfp::BatchTune tuned{};
  std::vector<hfp_ctx*> prep;     // helper contexts of the pair preparation threads
};

namespace hfp {

// One network of a batched FlowCutter launch (batch.cu).
struct BatchItem {
  hfp_net* net = nullptr;
  hfp_fc_params params{};
  int32_t* pierce_node_dev = nullptr;   // device piercing record (may be null)
  int8_t* pierce_side_dev = nullptr;
  int32_t pierce_cap = 0;
  hfp_fc_result result{};
  hfp_status status = HFP_OK;
  int32_t group_ctas = 0;          // CTAs of the group that solved it
};

// Inputs of the second construction algorithm (Section 6) for a block pair:
// H's vertex -> nets incidence (ascending), the nets' block masks, the pins
// of every (net, block) pair at cnt[noff[e] + rank of the block in mask[e]],
// and the pair's blocks (side 0 = b0, side 1 = b1).
struct SortBuildIn {
  const uint32_t* vnet_off;
  const int32_t* vnet;
  const unsigned long long* mask;
  const unsigned* noff;
  const unsigned* cnt;
  int32_t b0, b1;
};

// hfp_build_flow_network with optional restrictions (device inputs only):
// nets[n_nets] (ascending) holds every net of H with a pin in the region, and
// verts[n_verts] every vertex whose side is 0 or 1; only those are scanned.
// Null lists scan all of H.  With sb (and distances given) the nets come from
// the region's incidences sorted by net instead (the second construction
// algorithm); the network is the same.
hfp_status build_network_impl(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                              const int32_t* region, int32_t n_region, const int32_t* side,
                              const int32_t* dist_from_cut, const int32_t* nets, int32_t n_nets,
                              const int32_t* verts, int32_t n_verts, hfp_net** out,
                              const SortBuildIn* sb = nullptr);

// A helper context of `parent` for another host thread: the same device and
// tuning, a non-blocking stream of its own that is destroyed with it
// (hfp_ctx_destroy).  ctx_copy_tuning refreshes its tuning from the parent.
hfp_status ctx_fork(hfp_ctx* parent, hfp_ctx** out);
void ctx_copy_tuning(hfp_ctx* dst, const hfp_ctx* src);
// Moves a network to context `to` (its later work and frees go to `to`'s
// stream).  Every operation on the network's old stream must have finished.
void net_rehome(hfp_net* net, hfp_ctx* to);

// Allocates the buffers of one-phase rounds (P.fused_rounds) and queue-driven
// global relabels (P.async_gr) that the network does not have yet (api.cu).
hfp_status ensure_engine_buffers(hfp_net* net, const Params& P);

// Grid of fc_batch_kernel on the context's device (all CTAs co-resident).
hfp_status batch_grid(hfp_ctx* ctx, int* grid);
// Runs FlowCutter on every item in one launch; group_ctas <= 0 picks the
// largest group size that gives every item its own group.  ms_out (may be
// null) receives the kernel time.
hfp_status run_fc_batch(hfp_ctx* ctx, BatchItem* items, int n, int group_ctas, float* ms_out,
                        const BatchTune* tune = nullptr);

}  // namespace hfp
