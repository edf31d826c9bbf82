// Host implementation of the C ABI declared in include/hfp.h.
//
// The host only allocates, launches and reads back a few words: network
// construction, the push-relabel rounds, global relabels, residual BFSs and
// piercing all run in the kernels of build.cu, engine.cu and cuts.cu.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

using namespace hfp;

namespace hfp {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches_total() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hfp

namespace hfp {

namespace {
thread_local std::string g_err;
}  // namespace

hfp_status fail(hfp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

// error message setter for entry points defined in other translation units
void set_last_error(const char* msg) { g_err = msg; }

// Buffers only the one-phase rounds and the queue-driven global relabels
// use, allocated at the network's first launch that needs them.
hfp_status ensure_engine_buffers(hfp_net* net, const Params& P) {
  hfp_ctx* c = net->ctx;
  NetDev& D = net->d;
  const size_t NL = (size_t)D.NL;
  if (P.fused_rounds && !D.delta1) {
    CK(cudaMallocAsync(&net->delta1_buf, sizeof(long long) * (NL ? NL : 1), c->stream));
    CK(cudaMemsetAsync(net->delta1_buf, 0, sizeof(long long) * (NL ? NL : 1), c->stream));
    D.delta1 = (long long*)net->delta1_buf;
  }
  if (P.parpr_block && P.fused_rounds && !D.blk) {
    CK(cudaMallocAsync(&net->blk_buf, sizeof(uint32_t) * (NL ? NL : 1), c->stream));
    CK(cudaMemsetAsync(net->blk_buf, 0, sizeof(uint32_t) * (NL ? NL : 1), c->stream));
    D.blk = (uint32_t*)net->blk_buf;
  }
  // Work queue of the global relabel: room for every node's chunks four
  // times (a node is queued again whenever its label drops; the sinks of a
  // relabel after sink-side piercings are all seeds); a fuller queue makes
  // that relabel fall back to the level-by-level search.  Entries hold
  // 27-bit Lawler ids: larger networks relabel level by level.
  if (P.async_gr && !D.gq && D.NL < (1 << 27) - 1) {
    const uint64_t cap64 = 4 * ((uint64_t)D.NL + (uint64_t)D.p_pins / 8) + 4096;
    const unsigned cap = cap64 < 0xF0000000ull ? (unsigned)cap64 : 0xF0000000u;
    CK(cudaMallocAsync(&net->gq_buf, sizeof(unsigned long long) * cap, c->stream));
    CK(cudaMemsetAsync(net->gq_buf, 0, sizeof(unsigned long long) * cap, c->stream));   // empty
    D.gq = (unsigned long long*)net->gq_buf;
    D.gq_cap = cap;
  }
  return HFP_OK;
}

}  // namespace hfp

namespace {

int map_dev_err(int e) {
  switch (e) {
    case kDevOk: return HFP_OK;
    case kDevBadInput: return HFP_ERR_INVALID;
    default: return HFP_ERR_ITER_LIMIT;
  }
}

}  // namespace

namespace {

hfp_status set_device(hfp_ctx* ctx) {
  CK(cudaSetDevice(ctx->device));
  return HFP_OK;
}

hfp_status read_ctl(hfp_net* net, Ctl* out) {
  hfp_ctx* c = net->ctx;
  CK(cudaMemcpyAsync(c->pinned_ctl, &net->E->c, sizeof(Ctl), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *out = *c->pinned_ctl;
  return HFP_OK;
}

hfp_status run_engine(hfp_net* net) {
  hfp_ctx* c = net->ctx;
  Params P = c->params;
  if (hfp_status s0 = ensure_engine_buffers(net, P)) return s0;
  // without its buffers the engine runs the two-phase, level-by-level forms
  if (!net->d.delta1) P.fused_rounds = 0;
  if (!net->d.gq) P.async_gr = 0;
  if (!net->d.blk) P.parpr_block = 0;
  // flows after a piercing are incremental: their own stall rule
  if (net->pierced) {
    if (P.stall_rounds_pierce) P.stall_rounds = P.stall_rounds_pierce;
    else P.stall_adapt = 1;
  }
  void* args[] = {(void*)&net->d, (void*)&net->E, (void*)&P};
  CK(cudaEventRecord(c->ev0, c->stream));
  CK(cudaLaunchCooperativeKernel((void*)engine_kernel, dim3(c->coop_grid), dim3(c->threads),
                                 args, 0, c->stream));
  CK(cudaEventRecord(c->ev1, c->stream));
  count_launches(1);
  net->launches++;
  Ctl ctl;
  hfp_status s = read_ctl(net, &ctl);
  if (s != HFP_OK) return s;
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  net->engine_ns += (uint64_t)((double)ms * 1e6);
  if (ctl.err != kDevOk)
    return fail(map_dev_err(ctl.err), "flow engine stopped: device code %d (where %d)", ctl.err,
                ctl.err_where);
  return HFP_OK;
}

hfp_status stage_nodes(hfp_net* net, const int32_t* nodes, int32_t count) {
  hfp_ctx* c = net->ctx;
  if (count > net->dev_nodes_cap) {
    if (net->dev_nodes) CK(cudaFreeAsync(net->dev_nodes, c->stream));
    net->dev_nodes = nullptr;
    int32_t cap = count < 64 ? 64 : count;
    CK(cudaMallocAsync((void**)&net->dev_nodes, sizeof(int32_t) * cap, c->stream));
    net->dev_nodes_cap = cap;
  }
  for (int32_t i = 0; i < count; i++)
    if (nodes[i] < 0 || nodes[i] >= net->d.n_nodes)
      return fail(HFP_ERR_INVALID, "pierced node %d out of range", nodes[i]);
  if (count > 0) {
    CK(cudaMemcpyAsync(net->dev_nodes, nodes, sizeof(int32_t) * count, cudaMemcpyHostToDevice,
                       c->stream));
  }
  return HFP_OK;
}

// Flow from {s} at the first call: saturate s, then a global relabel seeds
// exact labels and the frontier; the engine runs to a maximum preflow and
// ends with a final global relabel (exact labels, T_r).
hfp_status ensure_max_flow(hfp_net* net) {
  if (net->labels_exact) return HFP_OK;
  hfp_ctx* c = net->ctx;
  if (!net->flow_started) {
    int32_t zero = 0;
    hfp_status s = stage_nodes(net, &zero, 1);
    if (s != HFP_OK) return s;
    launch_engine_setup(net->E, SETUP_PREP, c->stream);
    launch_saturate(net->d, net->E, net->dev_nodes, 1, c->stream);
    net->flow_started = true;
  }
  launch_engine_setup(net->E, SETUP_GR, c->stream);
  hfp_status s = run_engine(net);
  if (s != HFP_OK) return s;
  net->labels_exact = true;
  net->sr_valid = false;
  return HFP_OK;
}

hfp_status ensure_source_side(hfp_net* net) {
  if (net->sr_valid) return HFP_OK;
  if (net->sr_seed >= 0) launch_engine_setup(net->E, SETUP_SR_ADD, net->ctx->stream, net->sr_seed);
  else launch_engine_setup(net->E, SETUP_SR, net->ctx->stream);
  hfp_status s = run_engine(net);
  if (s != HFP_OK) return s;
  net->sr_valid = true;
  net->sr_seed = -1;
  return HFP_OK;
}

hfp_status ensure_dist(hfp_net* net) {
  if (net->dist_ready) return HFP_OK;
  launch_engine_setup(net->E, SETUP_DIST, net->ctx->stream);
  hfp_status s = run_engine(net);
  if (s != HFP_OK) return s;
  net->dist_ready = true;
  return HFP_OK;
}

hfp_status copy_out(void* dst, const void* src, size_t bytes, hfp_mem mem, cudaStream_t st) {
  CK(cudaMemcpyAsync(dst, src, bytes,
                     mem == HFP_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     st));
  return HFP_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
HFP_API const char* hfp_last_error(void) { return hfp::g_err.c_str(); }

HFP_API uint64_t hfp_kernel_launches(void) { return launches_total(); }

HFP_API hfp_status hfp_ctx_create(hfp_ctx** out, int device, void* stream) {
  if (!out) return fail(HFP_ERR_INVALID, "ctx pointer is NULL");
  *out = nullptr;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(HFP_ERR_INVALID, "no CUDA device %d", device);
  CK(cudaSetDevice(device));
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device));
  if (!coop) return fail(HFP_ERR_CUDA, "device %d lacks cooperative launch", device);
  hfp_ctx* c = new hfp_ctx();
  c->device = device;
  c->stream = (cudaStream_t)stream;
  cudaError_t e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  int per_sm = 0;
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel, c->threads, 0);
  if (e == cudaSuccess && per_sm < 1) e = cudaErrorInvalidConfiguration;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->pinned_ctl, sizeof(Ctl));
  if (e == cudaSuccess) e = cudaMallocHost(&c->pinned_small, 4096);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e != cudaSuccess) {
    if (c->pinned_ctl) cudaFreeHost(c->pinned_ctl);
    delete c;
    return fail(HFP_ERR_CUDA, "context set-up failed: %s", cudaGetErrorString(e));
  }
  if (per_sm > 2) per_sm = 2;
  c->coop_grid = c->sms * per_sm;
  c->params.timeout_ns = 10ull * 1000 * 1000 * 1000;
  c->params.max_rounds = 1ull << 22;
  c->params.gr_work = 0;           // set per network (a multiple of its node count)
  c->params.stall_rounds = 100;    // Section 8.3, "Avoid Pushing Flow Back" (tuned: 500 in the paper)
  c->params.stall_nodes = 1500;
  c->params.tail_enter = 64;       // CTA 0 alone at or below this frontier size
  c->params.tail_exit = 192;
  c->params.bfs_enter = 0;         // CTA 0 alone for BFS levels up to this size: off (the
  c->params.bfs_exit = 0;          // relabel BFS levels are wide; measured slower alone)
  c->params.pierce_relabel = 0;
  c->params.stall_rounds_pierce = 0;    // incremental flows after a piercing: adaptive
  c->params.stall_adapt = 0;
  c->params.async_gr = 1;          // global relabels as one queue-driven search
  c->params.gr_warps = 12;         // warps per CTA serving its queue (fewer: less re-expansion)
  c->params.fused_rounds = 1;      // one phase per discharge round
  *out = c;
  return HFP_OK;
}

// A context is freed when its caller has destroyed it and no network built
// from it is alive any more.
static void ctx_release(hfp_ctx* c) {
  if (c->refs.fetch_sub(1) != 1) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->owns_stream) cudaStreamDestroy(c->stream);
  if (c->pinned_ctl) cudaFreeHost(c->pinned_ctl);
  if (c->pinned_small) cudaFreeHost(c->pinned_small);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  delete c;
}

HFP_API void hfp_ctx_destroy(hfp_ctx* c) {
  if (c) ctx_release(c);
}

namespace hfp {

void ctx_copy_tuning(hfp_ctx* dst, const hfp_ctx* src) {
  dst->params = src->params;
  dst->gr_work_x100 = src->gr_work_x100;
  dst->batch_cluster = src->batch_cluster;
  dst->batch_big_ctas = src->batch_big_ctas;
  dst->batch_big_groups = src->batch_big_groups;
  dst->identical_nets = src->identical_nets;
  dst->batch_fused_rounds = src->batch_fused_rounds;
  dst->batch_async_gr = src->batch_async_gr;
  dst->construction = src->construction;
  dst->batch_gr_work_x100 = src->batch_gr_work_x100;
  dst->batch_stall_rounds_pierce = src->batch_stall_rounds_pierce;
  dst->prep_streams = src->prep_streams;
}

hfp_status ctx_fork(hfp_ctx* parent, hfp_ctx** out) {
  *out = nullptr;
  CK(cudaSetDevice(parent->device));
  cudaStream_t s = nullptr;
  CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  hfp_ctx* c = nullptr;
  const hfp_status r = hfp_ctx_create(&c, parent->device, (void*)s);
  if (r != HFP_OK) {
    cudaStreamDestroy(s);
    return r;
  }
  c->owns_stream = true;
  ctx_copy_tuning(c, parent);
  *out = c;
  return HFP_OK;
}

void net_rehome(hfp_net* net, hfp_ctx* to) {
  if (!net || net->ctx == to) return;
  to->refs.fetch_add(1);
  hfp_ctx* from = net->ctx;
  net->ctx = to;
  ctx_release(from);
}

}  // namespace hfp

HFP_API void hfp_net_destroy(hfp_net* net) {
  if (!net) return;
  hfp_ctx* c = net->ctx;
  cudaSetDevice(c->device);
  cudaStream_t st = c->stream;
  if (net->arena) cudaFreeAsync(net->arena, st);
  if (net->dev_nodes) cudaFreeAsync(net->dev_nodes, st);
  if (net->trace_buf) cudaFreeAsync(net->trace_buf, st);
  if (net->gq_buf) cudaFreeAsync(net->gq_buf, st);
  if (net->delta1_buf) cudaFreeAsync(net->delta1_buf, st);
  if (net->net_done_buf) cudaFreeAsync(net->net_done_buf, st);
  if (net->blk_buf) cudaFreeAsync(net->blk_buf, st);
  cudaStreamSynchronize(st);
  delete net;
  ctx_release(c);
}

namespace hfp {

hfp_status build_network_impl(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                              const int32_t* region, int32_t n_region, const int32_t* side,
                              const int32_t* dist_from_cut, const int32_t* nets, int32_t n_nets,
                              const int32_t* verts, int32_t n_verts, hfp_net** out,
                              const SortBuildIn* sb) {
  if (!out) return fail(HFP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!ctx || !H) return fail(HFP_ERR_INVALID, "ctx or H is NULL");
  const int32_t n = H->n, m = H->m;
  if (n < 0 || m < 0 || n_region < 0 || n_region > n)
    return fail(HFP_ERR_INVALID, "bad sizes n=%d m=%d n_region=%d", n, m, n_region);
  if (!H->net_off || (m > 0 && (!H->pins || !H->net_w)) || (n > 0 && !side) ||
      (n_region > 0 && !region))
    return fail(HFP_ERR_INVALID, "missing input array");
  if (mem != HFP_MEM_HOST && mem != HFP_MEM_DEVICE) return fail(HFP_ERR_INVALID, "bad mem");
  if ((nets || verts) && (mem != HFP_MEM_DEVICE || n_nets < 0 || n_verts < 0))
    return fail(HFP_ERR_INVALID, "net / vertex lists need device inputs");
  hfp_status s = set_device(ctx);
  if (s != HFP_OK) return s;
  cudaStream_t st = ctx->stream;
  const int sms = ctx->sms;
  // nets scanned (and per-net scratch entries): the list, or all of H, or
  // the runs of the sorted region incidences
  int32_t M = nets ? n_nets : m;

  // total pins of H
  uint32_t P = 0;
  if (mem == HFP_MEM_HOST) {
    if (H->net_off[0] != 0) return fail(HFP_ERR_INVALID, "net_off[0] != 0");
    for (int32_t e = 0; e < m; e++)
      if (H->net_off[e + 1] < H->net_off[e]) return fail(HFP_ERR_INVALID, "net_off decreases");
    P = H->net_off[m];
  } else {
    uint32_t* h = (uint32_t*)ctx->pinned_small;
    CK(cudaMemcpyAsync(h, H->net_off, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(h + 1, H->net_off + m, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (h[0] != 0) return fail(HFP_ERR_INVALID, "net_off[0] != 0");
    P = h[1];
  }
  if (P >= (1u << 31)) return fail(HFP_ERR_INVALID, "too many pins (%u)", P);

  // inputs on the device
  DevBuf in_off, in_pins, in_netw, in_nodew, in_side, in_region, in_dist;
  const uint32_t* d_off = H->net_off;
  const int32_t *d_pins = H->pins, *d_netw = H->net_w, *d_nodew = H->node_w, *d_side = side,
                *d_region = region, *d_dist = dist_from_cut;
  if (mem == HFP_MEM_HOST) {
    CK(in_off.alloc(sizeof(uint32_t) * (m + 1), st));
    CK(cudaMemcpyAsync(in_off.p, H->net_off, sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, st));
    d_off = in_off.as<uint32_t>();
    CK(in_pins.alloc(sizeof(int32_t) * P, st));
    if (P) CK(cudaMemcpyAsync(in_pins.p, H->pins, sizeof(int32_t) * P, cudaMemcpyHostToDevice, st));
    d_pins = in_pins.as<int32_t>();
    CK(in_netw.alloc(sizeof(int32_t) * m, st));
    if (m) CK(cudaMemcpyAsync(in_netw.p, H->net_w, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st));
    d_netw = in_netw.as<int32_t>();
    if (H->node_w) {
      CK(in_nodew.alloc(sizeof(int32_t) * n, st));
      if (n) CK(cudaMemcpyAsync(in_nodew.p, H->node_w, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
      d_nodew = in_nodew.as<int32_t>();
    }
    CK(in_side.alloc(sizeof(int32_t) * n, st));
    if (n) CK(cudaMemcpyAsync(in_side.p, side, sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
    d_side = in_side.as<int32_t>();
    CK(in_region.alloc(sizeof(int32_t) * n_region, st));
    if (n_region)
      CK(cudaMemcpyAsync(in_region.p, region, sizeof(int32_t) * n_region, cudaMemcpyHostToDevice, st));
    d_region = in_region.as<int32_t>();
    if (dist_from_cut) {
      CK(in_dist.alloc(sizeof(int32_t) * n_region, st));
      if (n_region)
        CK(cudaMemcpyAsync(in_dist.p, dist_from_cut, sizeof(int32_t) * n_region,
                           cudaMemcpyHostToDevice, st));
      d_dist = in_dist.as<int32_t>();
    }
  }

  // second construction algorithm: the region's (net, vertex) pairs sorted by
  // net; every run is a net of the region
  const bool use_sb = sb && dist_from_cut && mem == HFP_MEM_DEVICE;
  DevBuf sb_pos, sb_key, sb_val, sb_key2, sb_val2, sb_hist, sb_head, sb_rid, sb_rs, sb_rn, sb_scr,
      sb_tot;
  unsigned sb_R = 0;
  if (use_sb) {
    const size_t nr1 = (size_t)(n_region > 0 ? n_region : 1);
    CK(sb_pos.alloc(sizeof(unsigned) * nr1, st));
    CK(sb_tot.alloc(sizeof(unsigned), st));
    CK(sb_scr.alloc(sizeof(unsigned) * (scan_scratch_words((unsigned)nr1) + 8), st));
    unsigned P2 = 0;
    CK(sort_build_count(n_region, d_region, sb->vnet_off, sb_pos.as<unsigned>(),
                        sb_scr.as<unsigned>(), sb_tot.as<unsigned>(), &P2, sms, st));
    const size_t p2 = P2 > 0 ? P2 : 1;
    const unsigned T = (P2 + 511) / 512;
    const size_t hw = (size_t)256 * (T > 0 ? T : 1);
    CK(sb_key.alloc(sizeof(unsigned) * p2, st));
    CK(sb_val.alloc(sizeof(int32_t) * p2, st));
    CK(sb_key2.alloc(sizeof(unsigned) * p2, st));
    CK(sb_val2.alloc(sizeof(int32_t) * p2, st));
    CK(sb_head.alloc(sizeof(unsigned) * p2, st));
    CK(sb_rid.alloc(sizeof(unsigned) * p2, st));
    CK(sb_hist.alloc(sizeof(unsigned) * hw, st));
    CK(sb_rs.alloc(sizeof(unsigned) * (p2 + 1), st));
    CK(sb_rn.alloc(sizeof(int32_t) * p2, st));
    DevBuf scr2;
    CK(scr2.alloc(sizeof(unsigned) * (scan_scratch_words((unsigned)(p2 > hw ? p2 : hw)) + 8), st));
    CK(sort_build_runs(n_region, d_region, sb->vnet_off, sb->vnet, m, P2, sb_pos.as<unsigned>(),
                       scr2.as<unsigned>(), sb_tot.as<unsigned>(), sb_key.as<unsigned>(),
                       sb_val.as<int32_t>(), sb_key2.as<unsigned>(), sb_val2.as<int32_t>(),
                       sb_hist.as<unsigned>(), sb_head.as<unsigned>(), sb_rid.as<unsigned>(),
                       sb_rs.as<unsigned>(), sb_rn.as<int32_t>(), &sb_R, sms, st));
    M = (int32_t)sb_R;
  }

  // pass 1 scratch
  const int32_t n_nodes = n_region + 2;
  DevBuf loc, keep, size, has_s, has_t, net_pos, pin_pos, s_pos, t_pos, totals, wsum, err,
      dist_tmp, scan_scr;
  const size_t mm = (size_t)(M > 0 ? M : 1);
  CK(loc.alloc(sizeof(int32_t) * (n > 0 ? n : 1), st));
  CK(keep.alloc(sizeof(unsigned) * mm, st));
  CK(size.alloc(sizeof(unsigned) * mm, st));
  CK(has_s.alloc(sizeof(unsigned) * mm, st));
  CK(has_t.alloc(sizeof(unsigned) * mm, st));
  CK(net_pos.alloc(sizeof(unsigned) * mm, st));
  CK(pin_pos.alloc(sizeof(unsigned) * mm, st));
  CK(s_pos.alloc(sizeof(unsigned) * mm, st));
  CK(t_pos.alloc(sizeof(unsigned) * mm, st));
  CK(totals.alloc(sizeof(unsigned) * 8, st));
  CK(wsum.alloc(sizeof(unsigned long long) * 8, st));
  CK(err.alloc(sizeof(int), st));
  CK(dist_tmp.alloc(sizeof(int32_t) * (n_region > 0 ? n_region : 1), st));
  size_t scan_words = scan_scratch_words((unsigned)(M > n_nodes + 1 ? M : n_nodes + 1)) + 8;
  CK(scan_scr.alloc(sizeof(unsigned) * scan_words, st));
  if (n) CK(cudaMemsetAsync(loc.p, 0xFF, sizeof(int32_t) * n, st));
  CK(cudaMemsetAsync(totals.p, 0, sizeof(unsigned) * 8, st));
  CK(cudaMemsetAsync(wsum.p, 0, sizeof(unsigned long long) * 8, st));
  CK(cudaMemsetAsync(err.p, 0, sizeof(int), st));
  if (n_region) CK(cudaMemsetAsync(dist_tmp.p, 0, sizeof(int32_t) * n_region, st));

  // per-hypernode attribute arrays live in the final arena; region_map
  // needs them now, so they are allocated first (sizes are known)
  DevBuf attrs;
  const size_t attr_bytes = align_up(sizeof(int32_t) * n_nodes) * 3 + align_up(n_nodes);
  CK(attrs.alloc(attr_bytes, st));
  int32_t* a_gid = attrs.as<int32_t>();
  int32_t* a_w = (int32_t*)((char*)attrs.p + align_up(sizeof(int32_t) * n_nodes));
  int8_t* a_orig = (int8_t*)((char*)attrs.p + 3 * align_up(sizeof(int32_t) * n_nodes));

  unsigned* tot = totals.as<unsigned>();
  launch_region_map(n, n_region, d_region, d_side, d_nodew, loc.as<int32_t>(), a_gid, a_w, a_orig,
                    err.as<int>(), st);
  launch_st_weight(verts ? n_verts : n, verts, loc.as<int32_t>(), d_side, d_nodew,
                   wsum.as<unsigned long long>(), err.as<int>(), sms, st);
  if (use_sb)
    launch_sb_eval(sb_R, sb_rs.as<unsigned>(), sb_rn.as<int32_t>(), sb_val.as<int32_t>(),
                   d_region, d_side, d_netw, sb->mask, sb->noff, sb->cnt, sb->b0, sb->b1,
                   keep.as<unsigned>(), size.as<unsigned>(), has_s.as<unsigned>(),
                   has_t.as<unsigned>(), wsum.as<unsigned long long>() + 3, sms, st);
  else
    launch_net_scan(n, M, nets, d_off, d_pins, d_netw, d_side, loc.as<int32_t>(),
                    keep.as<unsigned>(), size.as<unsigned>(), has_s.as<unsigned>(),
                    has_t.as<unsigned>(), dist_tmp.as<int32_t>(), d_dist ? 0 : 1,
                    wsum.as<unsigned long long>() + 3, err.as<int>(), sms, st);
  if (M) {
    CK(cudaMemcpyAsync(net_pos.p, keep.p, sizeof(unsigned) * M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(pin_pos.p, size.p, sizeof(unsigned) * M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(s_pos.p, has_s.p, sizeof(unsigned) * M, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(t_pos.p, has_t.p, sizeof(unsigned) * M, cudaMemcpyDeviceToDevice, st));
  }
  scan_exclusive(net_pos.as<unsigned>(), M, scan_scr.as<unsigned>(), tot + 0, st);
  scan_exclusive(pin_pos.as<unsigned>(), M, scan_scr.as<unsigned>(), tot + 1, st);
  scan_exclusive(s_pos.as<unsigned>(), M, scan_scr.as<unsigned>(), tot + 2, st);
  scan_exclusive(t_pos.as<unsigned>(), M, scan_scr.as<unsigned>(), tot + 3, st);

  struct Head {
    unsigned totals[8];
    unsigned long long wsum[8];
    int err;
  };
  Head* hh = (Head*)ctx->pinned_small;
  CK(cudaMemcpyAsync(hh->totals, totals.p, sizeof(unsigned) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(hh->wsum, wsum.p, sizeof(unsigned long long) * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&hh->err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (hh->err != kDevOk) return fail(HFP_ERR_INVALID, "invalid hypergraph, region or side input");
  if (hh->wsum[2] >= (1ull << 31)) return fail(HFP_ERR_INVALID, "vertex weights sum to >= 2^31");
  if (hh->wsum[3] >= (1ull << 31)) return fail(HFP_ERR_INVALID, "net weights sum to >= 2^31");
  int32_t m_net = (int32_t)hh->totals[0];
  unsigned p_net = hh->totals[1];
  const int64_t NL64 = (int64_t)n_nodes + 2 * (int64_t)m_net;
  if (NL64 >= (1ll << 31) - 2) return fail(HFP_ERR_INVALID, "flow network too large");
  int32_t NL = (int32_t)NL64;
  // W of the flow problem: c(s) + c(t) + c(B)
  const int64_t total_w = (int64_t)hh->wsum[0] + (int64_t)hh->wsum[1] + (int64_t)hh->wsum[4];

  // arena for the network and its flow state
  hfp_net* net = new hfp_net();
  net->ctx = ctx;
  ctx->refs.fetch_add(1);
  net->n_region = n_region;
  std::vector<size_t> sz = {
      sizeof(uint32_t) * (m_net + 1), sizeof(int32_t) * p_net, sizeof(int32_t) * m_net,
      sizeof(int32_t) * m_net, sizeof(uint32_t) * (n_nodes + 1), sizeof(int2) * p_net,
      sizeof(int32_t) * n_nodes, sizeof(int32_t) * n_nodes, (size_t)n_nodes, sizeof(int32_t) * n_nodes,
      sizeof(int32_t) * p_net, sizeof(int32_t) * p_net, sizeof(int32_t) * m_net,
      sizeof(int32_t) * NL, sizeof(int32_t) * NL, sizeof(long long) * NL, sizeof(long long) * NL,
      sizeof(uint32_t) * NL, (size_t)NL, (size_t)NL, (size_t)NL, sizeof(int32_t) * NL,
      sizeof(int32_t) * NL, sizeof(int32_t) * NL, sizeof(int32_t) * NL, sizeof(EngineCtl)};
  size_t total = 0;
  for (size_t b : sz) total += align_up(b);
  cudaError_t ae = cudaMallocAsync(&net->arena, total, st);
  if (ae != cudaSuccess) {
    net->arena = nullptr;
    hfp_net_destroy(net);
    return fail(HFP_ERR_OOM, "cannot allocate %zu bytes for the flow network", total);
  }
  std::vector<char*> ptr;
  {
    char* q = (char*)net->arena;
    for (size_t b : sz) {
      ptr.push_back(q);
      q += align_up(b);
    }
  }
  NetDev& D = net->d;
  D.n_nodes = n_nodes;
  D.m_nets = m_net;
  D.NL = NL;
  D.p_pins = p_net;
  uint32_t* nnet_off = (uint32_t*)ptr[0];
  int32_t* npin = (int32_t*)ptr[1];
  int32_t* nnet_w = (int32_t*)ptr[2];
  net->net_gid = (int32_t*)ptr[3];
  unsigned* node_off = (unsigned*)ptr[4];
  int2* inc = (int2*)ptr[5];
  int32_t* node_w = (int32_t*)ptr[6];
  int32_t* node_dist = (int32_t*)ptr[7];
  int8_t* node_orig = (int8_t*)ptr[8];
  int32_t* node_gid = (int32_t*)ptr[9];
  D.net_off = nnet_off;
  D.pin = npin;
  D.net_w = nnet_w;
  D.node_off = node_off;
  D.inc = inc;
  D.node_w = node_w;
  D.node_dist = node_dist;
  D.node_orig = node_orig;
  D.node_gid = node_gid;
  D.f_in = (int32_t*)ptr[10];
  D.f_out = (int32_t*)ptr[11];
  D.f_b = (int32_t*)ptr[12];
  D.lab0 = (int32_t*)ptr[13];
  D.lab1 = (int32_t*)ptr[14];
  D.excess = (long long*)ptr[15];
  D.delta = (long long*)ptr[16];
  D.stamp = (uint32_t*)ptr[17];
  D.flags = (uint8_t*)ptr[18];
  D.needrl = (uint8_t*)ptr[19];
  D.insr = (uint8_t*)ptr[20];
  for (int k = 0; k < 4; k++) D.list[k] = (int32_t*)ptr[21 + k];
  net->E = (EngineCtl*)ptr[25];
  net->total_w = total_w;

  hfp_status rs = HFP_OK;
  auto done = [&](hfp_status r) {
    if (r != HFP_OK) hfp_net_destroy(net);
    return r;
  };
#define CKN(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return done(fail(HFP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_)));    \
  } while (0)

  CKN(cudaMemcpyAsync(node_gid, a_gid, sizeof(int32_t) * n_nodes, cudaMemcpyDeviceToDevice, st));
  CKN(cudaMemcpyAsync(node_w, a_w, sizeof(int32_t) * n_nodes, cudaMemcpyDeviceToDevice, st));
  CKN(cudaMemcpyAsync(node_orig, a_orig, n_nodes, cudaMemcpyDeviceToDevice, st));
  CKN(cudaMemsetAsync(D.flags, 0, NL, st));
  launch_st_attrs(node_gid, node_w, node_orig, wsum.as<unsigned long long>(), D.flags,
                  err.as<int>(), st);
  if (use_sb)
    launch_sb_fill(sb_R, sb_rs.as<unsigned>(), sb_rn.as<int32_t>(), sb_val.as<int32_t>(), d_side,
                   d_region, d_netw, keep.as<unsigned>(), net_pos.as<unsigned>(),
                   pin_pos.as<unsigned>(), s_pos.as<unsigned>(), t_pos.as<unsigned>(),
                   has_s.as<unsigned>(), has_t.as<unsigned>(), tot, nnet_off, npin, nnet_w,
                   net->net_gid, inc, sms, st);
  else
    launch_net_fill(M, nets, d_off, d_pins, d_netw, loc.as<int32_t>(), keep.as<unsigned>(),
                    net_pos.as<unsigned>(), pin_pos.as<unsigned>(), s_pos.as<unsigned>(),
                    t_pos.as<unsigned>(), has_s.as<unsigned>(), has_t.as<unsigned>(), tot,
                    nnet_off, npin, nnet_w, net->net_gid, inc, sms, st);
  {
    uint32_t* hp = (uint32_t*)((char*)ctx->pinned_small + 1024);
    *hp = p_net;
    CKN(cudaMemcpyAsync(nnet_off + m_net, hp, sizeof(uint32_t), cudaMemcpyHostToDevice, st));
  }
  // identical net removal (Section 6): the kept nets are compacted in place;
  // the incidence lists below are built from them (s / t lists from the
  // membership flags of the kept nets)
  DevBuf d_keep, d_newe, d_hs, d_ht, d_ps, d_pt;
  const int32_t m_before = m_net;
  const bool dedup = ctx->identical_nets && m_net > 1;
  if (dedup) {
    const int32_t m = m_net;
    unsigned tsz = 1;
    while (tsz < 2u * (unsigned)m) tsz <<= 1;
    DevBuf tag, ttag, tmin, rep, wacc, size, newp, o_off, o_pin, o_w, o_gid, sums;
    CKN(tag.alloc(sizeof(unsigned long long) * m, st));
    CKN(ttag.alloc(sizeof(unsigned long long) * tsz, st));
    CKN(tmin.alloc(sizeof(int32_t) * tsz, st));
    CKN(rep.alloc(sizeof(int32_t) * m, st));
    CKN(wacc.alloc(sizeof(unsigned long long) * m, st));
    CKN(d_keep.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(d_newe.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(size.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(newp.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(d_hs.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(d_ht.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(d_ps.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(d_pt.alloc(sizeof(unsigned) * (m + 1), st));
    CKN(sums.alloc(sizeof(unsigned) * 8, st));
    CKN(o_off.alloc(sizeof(uint32_t) * (m + 1), st));
    CKN(o_pin.alloc(sizeof(int32_t) * (p_net > 0 ? p_net : 1), st));
    CKN(o_w.alloc(sizeof(int32_t) * m, st));
    CKN(o_gid.alloc(sizeof(int32_t) * m, st));
    CKN(cudaMemsetAsync(ttag.p, 0, sizeof(unsigned long long) * tsz, st));
    CKN(cudaMemsetAsync(tmin.p, 0x7f, sizeof(int32_t) * tsz, st));
    CKN(cudaMemsetAsync(wacc.p, 0, sizeof(unsigned long long) * m, st));
    launch_net_tags(m, nnet_off, npin, tag.as<unsigned long long>(),
                    ttag.as<unsigned long long>(), tmin.as<int32_t>(), tsz - 1, rep.as<int32_t>(),
                    err.as<int>(), sms, st);
    launch_net_merge(m, nnet_off, npin, nnet_w, rep.as<int32_t>(), wacc.as<unsigned long long>(),
                     d_keep.as<unsigned>(), size.as<unsigned>(), d_hs.as<unsigned>(),
                     d_ht.as<unsigned>(), sms, st);
    // exclusive scans: new net ids, new pin offsets, positions in the s / t lists
    CKN(cudaMemcpyAsync(d_newe.p, d_keep.p, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(newp.p, size.p, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(d_ps.p, d_hs.p, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(d_pt.p, d_ht.p, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, st));
    unsigned* sm = sums.as<unsigned>();
    scan_exclusive(d_newe.as<unsigned>(), m, scan_scr.as<unsigned>(), sm + 0, st);
    scan_exclusive(newp.as<unsigned>(), m, scan_scr.as<unsigned>(), sm + 1, st);
    scan_exclusive(d_ps.as<unsigned>(), m, scan_scr.as<unsigned>(), sm + 2, st);
    scan_exclusive(d_pt.as<unsigned>(), m, scan_scr.as<unsigned>(), sm + 3, st);
    launch_net_compact(m, nnet_off, npin, net->net_gid, d_keep.as<unsigned>(),
                       d_newe.as<unsigned>(), newp.as<unsigned>(),
                       wacc.as<unsigned long long>(), o_off.as<uint32_t>(), o_pin.as<int32_t>(),
                       o_w.as<int32_t>(), o_gid.as<int32_t>(), sms, st);
    unsigned* hs = (unsigned*)((char*)ctx->pinned_small + 1024);
    CKN(cudaMemcpyAsync(hs, sm, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CKN(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CKN(cudaStreamSynchronize(st));
    if (herr) return done(fail(HFP_ERR_CUDA, "identical net table overflow"));
    m_net = (int32_t)hs[0];
    p_net = hs[1];
    NL = n_nodes + 2 * m_net;
    CKN(cudaMemcpyAsync(nnet_off, o_off.p, sizeof(uint32_t) * m_net, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(npin, o_pin.p, sizeof(int32_t) * p_net, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(nnet_w, o_w.p, sizeof(int32_t) * m_net, cudaMemcpyDeviceToDevice, st));
    CKN(cudaMemcpyAsync(net->net_gid, o_gid.p, sizeof(int32_t) * m_net, cudaMemcpyDeviceToDevice,
                        st));
    launch_dedup_totals((unsigned)m_net, p_net, sm + 2, sm + 3, nnet_off, tot, st);
    D.m_nets = m_net;
    D.NL = NL;
    D.p_pins = p_net;
  }
  {
    DevBuf cursor, tmp;
    CKN(cursor.alloc(sizeof(unsigned) * n_nodes, st));
    CKN(tmp.alloc(sizeof(int2) * (p_net > 0 ? p_net : 1), st));
    launch_incidence(n_nodes, m_net, p_net, nnet_off, npin, node_off, cursor.as<unsigned>(), tot,
                     inc, tmp.as<int2>(), scan_scr.as<unsigned>(), tot + 4, sms, st);
  }
  if (dedup)
    launch_st_inc(m_before, nnet_off, d_keep.as<unsigned>(), d_newe.as<unsigned>(),
                  d_hs.as<unsigned>(), d_ht.as<unsigned>(), d_ps.as<unsigned>(),
                  d_pt.as<unsigned>(), node_off, nnet_off, inc, sms, st);
  launch_heavy_flags(D, sms, st);
  // distances from the original cut: given, or seeded here and completed by
  // the engine on first use (ensure_dist)
  if (d_dist) {
    launch_dist_copy(n_region, d_dist, node_dist, err.as<int>(), st);
    net->dist_ready = true;
  } else {
    launch_dist_seed(n_nodes, dist_tmp.as<int32_t>(), node_dist, sms, st);
    net->dist_ready = false;
  }
  // flow state
  CKN(cudaMemsetAsync(D.f_in, 0, sizeof(int32_t) * p_net, st));
  CKN(cudaMemsetAsync(D.f_out, 0, sizeof(int32_t) * p_net, st));
  CKN(cudaMemsetAsync(D.f_b, 0, sizeof(int32_t) * m_net, st));
  CKN(cudaMemsetAsync(D.excess, 0, sizeof(long long) * NL, st));
  CKN(cudaMemsetAsync(D.delta, 0, sizeof(long long) * NL, st));
  CKN(cudaMemsetAsync(D.stamp, 0, sizeof(uint32_t) * NL, st));
  CKN(cudaMemsetAsync(D.needrl, 0, NL, st));
  CKN(cudaMemsetAsync(D.insr, 0, NL, st));
  {
    EngineCtl* h = (EngineCtl*)((char*)ctx->pinned_small + 2048 + 64);
    static_assert(sizeof(EngineCtl) + 2048 + 64 <= 4096, "staging too small");
    memset(h, 0, sizeof(EngineCtl));
    h->s.epoch = 1;
    h->s.state = ST_DONE;
    CKN(cudaMemcpyAsync(net->E, h, sizeof(EngineCtl), cudaMemcpyHostToDevice, st));
  }
  CKN(cudaMemcpyAsync(&hh->err, err.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKN(cudaStreamSynchronize(st));
  if (hh->err != kDevOk) return done(fail(HFP_ERR_INVALID, "invalid dist_from_cut input"));
  ctx->params.gr_work = 0;
  *out = net;
  return done(rs);
#undef CKN
}

}  // namespace hfp

HFP_API hfp_status hfp_build_flow_network(hfp_ctx* ctx, const hfp_hypergraph* H, hfp_mem mem,
                                          const int32_t* region, int32_t n_region,
                                          const int32_t* side, const int32_t* dist_from_cut,
                                          hfp_net** out) {
  return build_network_impl(ctx, H, mem, region, n_region, side, dist_from_cut, nullptr, 0,
                            nullptr, 0, out);
}

HFP_API hfp_status hfp_net_get_info(hfp_net* net, hfp_net_info* info) {
  if (!net || !info) return fail(HFP_ERR_INVALID, "NULL argument");
  info->n_nodes = net->d.n_nodes;
  info->m_nets = net->d.m_nets;
  info->p_pins = net->d.p_pins;
  info->lawler_nodes = net->d.NL;
  info->pad = 0;
  info->total_weight = net->total_w;
  return HFP_OK;
}

HFP_API hfp_status hfp_net_export(hfp_net* net, hfp_mem mem, uint32_t* net_off, int32_t* pins,
                                  int32_t* net_w, int32_t* net_gid, int32_t* node_w,
                                  uint32_t* node_off, int32_t* inc_slot, int32_t* dist) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  cudaStream_t st = net->ctx->stream;
  const NetDev& D = net->d;
  if (net_off && (s = copy_out(net_off, D.net_off, sizeof(uint32_t) * (D.m_nets + 1), mem, st))) return s;
  if (pins && (s = copy_out(pins, D.pin, sizeof(int32_t) * D.p_pins, mem, st))) return s;
  if (net_w && (s = copy_out(net_w, D.net_w, sizeof(int32_t) * D.m_nets, mem, st))) return s;
  if (net_gid && (s = copy_out(net_gid, net->net_gid, sizeof(int32_t) * D.m_nets, mem, st))) return s;
  if (node_w && (s = copy_out(node_w, D.node_w, sizeof(int32_t) * D.n_nodes, mem, st))) return s;
  if (node_off && (s = copy_out(node_off, D.node_off, sizeof(uint32_t) * (D.n_nodes + 1), mem, st))) return s;
  if (dist) {
    if ((s = ensure_dist(net)) != HFP_OK) return s;
    DevBuf tmp;
    CK(tmp.alloc(sizeof(int32_t) * D.n_nodes, st));
    launch_dist_export(D.n_nodes, D.node_dist, tmp.as<int32_t>(), net->ctx->sms, st);
    if ((s = copy_out(dist, tmp.p, sizeof(int32_t) * D.n_nodes, mem, st))) return s;
  }
  if (inc_slot) {
    DevBuf tmp;
    CK(tmp.alloc(sizeof(int32_t) * (D.p_pins > 0 ? D.p_pins : 1), st));
    launch_inc_slots(D, tmp.as<int32_t>(), net->ctx->sms, st);
    if ((s = copy_out(inc_slot, tmp.p, sizeof(int32_t) * D.p_pins, mem, st))) return s;
  }
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}

HFP_API hfp_status hfp_net_export_flow(hfp_net* net, hfp_mem mem, int32_t* f_in, int32_t* f_out,
                                       int32_t* f_b, int64_t* excess, int64_t* delta,
                                       uint8_t* flags) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  cudaStream_t st = net->ctx->stream;
  const NetDev& D = net->d;
  const size_t p = (size_t)D.p_pins, m = (size_t)D.m_nets, nl = (size_t)D.NL;
  if (f_in && (s = copy_out(f_in, D.f_in, sizeof(int32_t) * p, mem, st))) return s;
  if (f_out && (s = copy_out(f_out, D.f_out, sizeof(int32_t) * p, mem, st))) return s;
  if (f_b && (s = copy_out(f_b, D.f_b, sizeof(int32_t) * m, mem, st))) return s;
  if (excess && (s = copy_out(excess, D.excess, sizeof(int64_t) * nl, mem, st))) return s;
  if (delta) {
    // both delta buffers (one-phase rounds alternate them)
    DevBuf tmp;
    CK(tmp.alloc(sizeof(int64_t) * (nl > 0 ? nl : 1), st));
    launch_add_i64(D.delta, D.delta1, tmp.as<long long>(), (long long)nl, net->ctx->sms, st);
    if ((s = copy_out(delta, tmp.p, sizeof(int64_t) * nl, mem, st))) return s;
  }
  if (flags && (s = copy_out(flags, D.flags, nl, mem, st))) return s;
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}

HFP_API hfp_status hfp_net_get_stats(hfp_net* net, hfp_stats* out) {
  if (!net || !out) return fail(HFP_ERR_INVALID, "NULL argument");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  out->rounds = c.rounds;
  out->global_relabels = c.global_relabels;
  out->gr_levels = c.gr_levels;
  out->gr_queue_entries = c.gq_items;
  out->gr_queue_overflows = c.gq_overs;
  out->items_hyper = c.items_hyper;
  out->items_net = c.items_net;
  out->node_visits = c.node_visits;
  out->pushes = c.pushes;
  out->engine_launches = net->launches;
  out->engine_ns = net->engine_ns;
  return HFP_OK;
}

HFP_API hfp_status hfp_net_enable_trace(hfp_net* net, int32_t phases) {
  if (!net || phases < 0) return fail(HFP_ERR_INVALID, "bad trace arguments");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  cudaStream_t st = net->ctx->stream;
  if (net->trace_buf) CK(cudaFreeAsync(net->trace_buf, st));
  net->trace_buf = nullptr;
  net->d.trace = nullptr;
  net->d.trace_cap = 0;
  if (phases > 0) {
    CK(cudaMallocAsync(&net->trace_buf, sizeof(unsigned long long) * 4 * (size_t)phases, st));
    net->d.trace = (unsigned long long*)net->trace_buf;
    net->d.trace_cap = (unsigned)phases;
  }
  CK(cudaMemsetAsync(&net->E->c.trace_len, 0, sizeof(unsigned long long), st));
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}

HFP_API hfp_status hfp_net_get_trace(hfp_net* net, uint64_t* state_ns, uint64_t* state_cnt,
                                     uint64_t* trace, int32_t cap, int32_t* n) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (state_ns) memcpy(state_ns, c.state_ns, sizeof(c.state_ns));
  if (state_cnt) memcpy(state_cnt, c.state_cnt, sizeof(c.state_cnt));
  int32_t len = (int32_t)c.trace_len;
  if (n) *n = len;
  if (trace && cap > 0 && len > 0 && net->trace_buf) {
    int32_t k = len < cap ? len : cap;
    CK(cudaMemcpy(trace, net->trace_buf, sizeof(unsigned long long) * 4 * (size_t)k,
                  cudaMemcpyDeviceToHost));
  }
  return HFP_OK;
}

static void set_gr_work(hfp_net* net) {
  // global relabel after work linear in the network (Section 8.1): once the
  // frontier and next-list entries processed since the last one exceed
  // gr_work_x100 / 100 times the number of Lawler nodes
  net->ctx->params.gr_work =
      (unsigned long long)net->d.NL * net->ctx->gr_work_x100 / 100 + 1024;
}

HFP_API hfp_status hfp_ctx_get_tuning(hfp_ctx* ctx, hfp_tuning* t) {
  if (!ctx || !t) return fail(HFP_ERR_INVALID, "NULL argument");
  t->gr_work_x100 = ctx->gr_work_x100;
  t->stall_rounds = (uint32_t)ctx->params.stall_rounds;
  t->stall_nodes = ctx->params.stall_nodes;
  t->tail_enter = ctx->params.tail_enter;
  t->tail_exit = ctx->params.tail_exit;
  t->max_rounds = (uint32_t)ctx->params.max_rounds;
  t->bfs_enter = ctx->params.bfs_enter;
  t->bfs_exit = ctx->params.bfs_exit;
  t->pierce_relabel = ctx->params.pierce_relabel;
  t->stall_rounds_pierce = (uint32_t)ctx->params.stall_rounds_pierce;
  t->async_gr = ctx->params.async_gr;
  t->gr_warps = ctx->params.gr_warps;
  t->fused_rounds = ctx->params.fused_rounds;
  t->identical_nets = ctx->identical_nets;
  t->batch_cluster = ctx->batch_cluster;
  t->batch_big_ctas = ctx->batch_big_ctas;
  t->batch_big_groups = ctx->batch_big_groups;
  t->batch_fused_rounds = ctx->batch_fused_rounds;
  t->batch_async_gr = ctx->batch_async_gr;
  t->parpr_block = ctx->params.parpr_block;
  t->construction = ctx->construction;
  t->batch_gr_work_x100 = ctx->batch_gr_work_x100;
  t->batch_stall_rounds_pierce = ctx->batch_stall_rounds_pierce;
  t->wait_timeout_ms = (uint32_t)(ctx->params.timeout_ns / 1000000ull);
  t->prep_streams = ctx->prep_streams;
  return HFP_OK;
}

HFP_API hfp_status hfp_ctx_set_tuning(hfp_ctx* ctx, const hfp_tuning* t) {
  if (!ctx || !t) return fail(HFP_ERR_INVALID, "NULL argument");
  if (t->gr_work_x100 == 0 || t->stall_rounds == 0 || t->max_rounds == 0 ||
      t->tail_exit < t->tail_enter || t->bfs_exit < t->bfs_enter || t->batch_gr_work_x100 == 0 ||
      t->wait_timeout_ms == 0 || t->wait_timeout_ms > 600000 || t->prep_streams == 0 ||
      t->prep_streams > 16)
    return fail(HFP_ERR_INVALID, "bad tuning values");
  ctx->gr_work_x100 = t->gr_work_x100;
  ctx->params.stall_rounds = t->stall_rounds;
  ctx->params.stall_nodes = t->stall_nodes;
  ctx->params.tail_enter = t->tail_enter;
  ctx->params.tail_exit = t->tail_exit;
  ctx->params.max_rounds = t->max_rounds;
  ctx->params.bfs_enter = t->bfs_enter;
  ctx->params.bfs_exit = t->bfs_exit;
  ctx->params.pierce_relabel = t->pierce_relabel ? 1 : 0;
  ctx->params.stall_rounds_pierce = t->stall_rounds_pierce;
  ctx->params.async_gr = t->async_gr ? 1 : 0;
  ctx->params.gr_warps = t->gr_warps < 1 ? 1 : (t->gr_warps > 16 ? 16 : t->gr_warps);
  ctx->params.fused_rounds = t->fused_rounds ? 1 : 0;
  ctx->identical_nets = t->identical_nets ? 1 : 0;
  ctx->batch_cluster = t->batch_cluster <= 2 ? t->batch_cluster : 1;
  ctx->batch_big_ctas = t->batch_big_ctas;
  ctx->batch_big_groups = t->batch_big_groups;
  ctx->batch_fused_rounds = t->batch_fused_rounds ? 1 : 0;
  ctx->batch_async_gr = t->batch_async_gr ? 1 : 0;
  ctx->params.parpr_block = t->parpr_block ? 1 : 0;
  ctx->construction = t->construction <= 2 ? t->construction : 1;
  ctx->batch_gr_work_x100 = t->batch_gr_work_x100;
  ctx->batch_stall_rounds_pierce = t->batch_stall_rounds_pierce;
  ctx->params.timeout_ns = (unsigned long long)t->wait_timeout_ms * 1000000ull;
  ctx->prep_streams = t->prep_streams;
  return HFP_OK;
}

HFP_API hfp_status hfp_max_flow(hfp_net* net, int64_t* flow_value) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  set_gr_work(net);
  if ((s = ensure_max_flow(net)) != HFP_OK) return s;
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (flow_value) *flow_value = (int64_t)c.flow;
  return HFP_OK;
}

HFP_API hfp_status hfp_min_cut_source_side(hfp_net* net, hfp_mem mem, uint8_t* in_source_lawler,
                                           uint8_t* in_source_region, int32_t* cut_nets,
                                           int32_t cap, int32_t* n_cut, int64_t* source_weight) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  if (!net->labels_exact) return fail(HFP_ERR_STATE, "hfp_max_flow has not completed");
  set_gr_work(net);
  if ((s = ensure_source_side(net)) != HFP_OK) return s;
  cudaStream_t st = net->ctx->stream;
  const NetDev& D = net->d;
  if (in_source_lawler && (s = copy_out(in_source_lawler, D.insr, D.NL, mem, st))) return s;
  if (in_source_region && net->n_region > 0 &&
      (s = copy_out(in_source_region, D.insr + 2, net->n_region, mem, st)))
    return s;
  hfp_status ret = HFP_OK;
  if (n_cut || cut_nets) {
    DevBuf flags, pos, total, scr, outbuf;
    const unsigned m = (unsigned)D.m_nets;
    CK(flags.alloc(sizeof(unsigned) * (m ? m : 1), st));
    CK(pos.alloc(sizeof(unsigned) * (m ? m : 1), st));
    CK(total.alloc(sizeof(unsigned), st));
    CK(scr.alloc(sizeof(unsigned) * (scan_scratch_words(m) + 8), st));
    launch_cut_net_flags(D, flags.as<unsigned>(), net->ctx->sms, st);
    if (m) CK(cudaMemcpyAsync(pos.p, flags.p, sizeof(unsigned) * m, cudaMemcpyDeviceToDevice, st));
    scan_exclusive(pos.as<unsigned>(), m, scr.as<unsigned>(), total.as<unsigned>(), st);
    unsigned* hc = (unsigned*)net->ctx->pinned_small;
    CK(cudaMemcpyAsync(hc, total.p, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int32_t nc = (int32_t)*hc;
    if (n_cut) *n_cut = nc;
    if (cut_nets && cap > 0) {
      int32_t* dst = cut_nets;
      if (mem == HFP_MEM_HOST) {
        CK(outbuf.alloc(sizeof(int32_t) * cap, st));
        dst = outbuf.as<int32_t>();
      }
      launch_cut_net_compact(D, flags.as<unsigned>(), pos.as<unsigned>(), net->net_gid, dst, cap,
                             net->ctx->sms, st);
      if (mem == HFP_MEM_HOST)
        CK(cudaMemcpyAsync(cut_nets, dst, sizeof(int32_t) * (nc < cap ? nc : cap),
                           cudaMemcpyDeviceToHost, st));
    }
    if (nc > cap && cut_nets) ret = fail(HFP_ERR_BUFFER_TOO_SMALL, "cut_nets needs %d entries", nc);
  }
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (source_weight) *source_weight = c.wS;
  return ret;
}

HFP_API hfp_status hfp_min_cut_sink_side(hfp_net* net, hfp_mem mem, uint8_t* in_sink_lawler,
                                         uint8_t* in_sink_region, int64_t* sink_weight) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  if (!net->labels_exact) return fail(HFP_ERR_STATE, "hfp_max_flow has not completed");
  cudaStream_t st = net->ctx->stream;
  const NetDev& D = net->d;
  if (in_sink_lawler || in_sink_region) {
    DevBuf tmp;
    CK(tmp.alloc(D.NL, st));
    launch_lawler_sink_side(D, tmp.as<uint8_t>(), net->ctx->sms, st);
    if (in_sink_lawler && (s = copy_out(in_sink_lawler, tmp.p, D.NL, mem, st))) return s;
    if (in_sink_region && net->n_region > 0 &&
        (s = copy_out(in_sink_region, tmp.as<uint8_t>() + 2, net->n_region, mem, st)))
      return s;
  }
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (sink_weight) *sink_weight = c.wT;
  return HFP_OK;
}

namespace {

// Piercing-node selection by the rule of Section 7 (see hfp_flowcutter):
// the candidate with the largest key, or with the largest key below `below`
// (the next one in key order after a pick) when below != 0; w_reach < 0
// takes the growing side's reachable weight.
hfp_status select_pierce(hfp_net* net, int grow_s, const hfp_fc_params* prm, int32_t* node,
                         bool* no_path = nullptr, long long w_reach = -1,
                         unsigned long long below = 0, unsigned long long* key = nullptr,
                         uint32_t seed_override = 0, bool use_seed = false) {
  Ctl c;
  hfp_status s = ensure_dist(net);
  if (s != HFP_OK) return s;
  s = read_ctl(net, &c);
  if (s != HFP_OK) return s;
  if (w_reach < 0) w_reach = grow_s ? c.wS : c.wT;
  launch_pierce_select(net->d, net->E, grow_s, prm->max_block_weight, w_reach,
                       use_seed ? seed_override : prm->seed, net->ctx->sms, net->ctx->stream,
                       below);
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (c.best_key == 0 || c.best_node < 0) {
    *node = -1;
    return fail(HFP_NO_BALANCED_CUT, "no piercing candidate");
  }
  *node = c.best_node;
  if (no_path) *no_path = ((c.best_key >> 53) & 1ull) != 0;
  if (key) *key = c.best_key;
  return HFP_OK;
}

// Piercing (Algorithm 2, the S or T update).  With `lazy` (one node that
// has no augmenting path) the flow is left alone: the current preflow stays
// a maximum preflow and the flow value does not change.
//  - Source side (node not in T_r): T_r stays and S_r only grows by what the
//    node reaches, so only the node is marked and the next source-side search
//    starts from it.  Its arcs stay unsaturated until a sink-side piercing
//    could open a path through them; a later source-side piercing makes all it
//    reaches sources anyway.
//  - Sink side (node not in S_r): S_r stays and T_r grows by the nodes that
//    reach it, found by a reverse search from it alone; the labels are then no
//    longer exact distances, so the next flow computation first relabels.
hfp_status pierce(hfp_net* net, int side, const int32_t* nodes, int32_t count,
                  bool lazy = false) {
  hfp_status s = stage_nodes(net, nodes, count);
  if (s != HFP_OK) return s;
  net->pierced = true;
  cudaStream_t st = net->ctx->stream;
  if (side == 0) {
    // S <- S_r + nodes; labels stay valid, the new excess is the frontier
    launch_mark_sources(net->d, net->E, net->dev_nodes, count, net->ctx->sms, st);
    if (lazy && count == 1) {
      net->pending_source = nodes[0];
      net->sr_seed = net->sr_valid ? nodes[0] : -1;
      net->sr_valid = false;
      return HFP_OK;
    }
    net->pending_source = -1;
    launch_engine_setup(net->E, SETUP_PREP, st);
    launch_saturate(net->d, net->E, net->dev_nodes, count, st);
    launch_engine_setup(net->E,
                        net->gr_pending || net->ctx->params.pierce_relabel ? SETUP_GR
                                                                           : SETUP_ROUND,
                        st);
  } else {
    // T <- T_r + nodes; labels are no longer lower bounds: relabel globally
    launch_mark_sinks(net->d, net->E, net->dev_nodes, count, net->ctx->sms, st);
    if (lazy && count == 1) {
      launch_engine_setup(net->E, SETUP_GR_ADD, st, nodes[0]);
      net->labels_exact = false;
      if ((s = run_engine(net)) != HFP_OK) return s;
      net->labels_exact = true;
      net->gr_pending = true;
      return HFP_OK;
    }
    if (net->pending_source >= 0) {
      // the unsaturated source may now reach T: saturate it before the flow
      const int32_t u = net->pending_source;
      net->pending_source = -1;
      if ((s = stage_nodes(net, &u, 1)) != HFP_OK) return s;
      launch_engine_setup(net->E, SETUP_PREP, st);
      launch_saturate(net->d, net->E, net->dev_nodes, 1, st);
    }
    launch_engine_setup(net->E, SETUP_GR, st);
  }
  net->labels_exact = false;
  net->sr_valid = false;
  net->sr_seed = -1;
  net->gr_pending = false;
  if ((s = run_engine(net)) != HFP_OK) return s;
  net->labels_exact = true;
  return HFP_OK;
}

}  // namespace

HFP_API hfp_status hfp_pierce_and_augment(hfp_net* net, int32_t side, const int32_t* nodes,
                                          int32_t count, const hfp_fc_params* params,
                                          int32_t* pierced, int64_t* flow_value) {
  if (!net) return fail(HFP_ERR_INVALID, "net is NULL");
  if (side != 0 && side != 1) return fail(HFP_ERR_INVALID, "side must be 0 or 1");
  if (nodes && count <= 0) return fail(HFP_ERR_INVALID, "count must be positive");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  set_gr_work(net);
  if (!net->labels_exact) return fail(HFP_ERR_STATE, "hfp_max_flow has not completed");
  if ((s = ensure_source_side(net)) != HFP_OK) return s;
  int32_t chosen = -1;
  if (!nodes) {
    if (!params) return fail(HFP_ERR_INVALID, "params needed to select a piercing node");
    if ((s = select_pierce(net, side == 0, params, &chosen)) != HFP_OK) return s;
    nodes = &chosen;
    count = 1;
  }
  if (pierced) *pierced = nodes[0];
  if ((s = pierce(net, side, nodes, count)) != HFP_OK) return s;
  Ctl c;
  if ((s = read_ctl(net, &c)) != HFP_OK) return s;
  if (flow_value) *flow_value = (int64_t)c.flow;
  return HFP_OK;
}

namespace {

// Device state a most-balanced-cut repetition starts from (the first
// balanced state): terminal flags, S_r marks, labels, excess and the control
// block (all but its stamp epoch, which keeps increasing), plus the
// host-side bookkeeping of the network.
struct NetSnapshot {
  DevBuf flags, insr, lab0, lab1, excess, ctl;
  int32_t pending_source, sr_seed;
  bool sr_valid, labels_exact, gr_pending, pierced;

  hfp_status take(hfp_net* net) {
    const NetDev& D = net->d;
    cudaStream_t st = net->ctx->stream;
    const size_t NL = (size_t)D.NL;
    CK(flags.alloc(NL, st));
    CK(insr.alloc(NL, st));
    CK(lab0.alloc(4 * NL, st));
    CK(lab1.alloc(4 * NL, st));
    CK(excess.alloc(8 * NL, st));
    CK(ctl.alloc(sizeof(EngineCtl), st));
    CK(cudaMemcpyAsync(flags.p, D.flags, NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(insr.p, D.insr, NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(lab0.p, D.lab0, 4 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(lab1.p, D.lab1, 4 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(excess.p, D.excess, 8 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(ctl.p, net->E, sizeof(EngineCtl), cudaMemcpyDeviceToDevice, st));
    pending_source = net->pending_source;
    sr_seed = net->sr_seed;
    sr_valid = net->sr_valid;
    labels_exact = net->labels_exact;
    gr_pending = net->gr_pending;
    pierced = net->pierced;
    return HFP_OK;
  }

  hfp_status restore(hfp_net* net) const {
    const NetDev& D = net->d;
    cudaStream_t st = net->ctx->stream;
    const size_t NL = (size_t)D.NL;
    // the stamp epoch moves on rather than back: stamps written since the
    // snapshot must not match the searches of the next repetition
    unsigned epoch = 0;
    CK(cudaMemcpyAsync(&epoch, &net->E->s.epoch, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaMemcpyAsync(D.flags, flags.p, NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(D.insr, insr.p, NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(D.lab0, lab0.p, 4 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(D.lab1, lab1.p, 4 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(D.excess, excess.p, 8 * NL, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(net->E, ctl.p, sizeof(EngineCtl), cudaMemcpyDeviceToDevice, st));
    unsigned* h = (unsigned*)((char*)net->ctx->pinned_small + 1024);
    *h = epoch + 1;
    CK(cudaMemcpyAsync(&net->E->s.epoch, h, sizeof(unsigned), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    net->pending_source = pending_source;
    net->sr_seed = sr_seed;
    net->sr_valid = sr_valid;
    net->labels_exact = labels_exact;
    net->gr_pending = gr_pending;
    net->pierced = pierced;
    return HFP_OK;
  }
};

hfp_status node_weight(hfp_net* net, int32_t h, int64_t* w) {
  int32_t v = 0;
  CK(cudaMemcpyAsync(&v, net->d.node_w + h, sizeof(int32_t), cudaMemcpyDeviceToHost,
                     net->ctx->stream));
  CK(cudaStreamSynchronize(net->ctx->stream));
  *w = v;
  return HFP_OK;
}

}  // namespace

HFP_API hfp_status hfp_flowcutter(hfp_net* net, const hfp_fc_params* prm, uint8_t* final_side,
                                  int32_t* pierce_side, int32_t* pierce_node, int32_t pierce_cap,
                                  hfp_fc_result* result) {
  if (!net || !prm) return fail(HFP_ERR_INVALID, "NULL argument");
  if (prm->bulk_beta_pct < 0 || prm->bulk_beta_pct > 100 || prm->bulk_warmup < 0 ||
      prm->mb_reps < 0 || prm->mb_reps > 1024)
    return fail(HFP_ERR_INVALID, "bad bulk piercing or most balanced cut parameters");
  hfp_status s = set_device(net->ctx);
  if (s != HFP_OK) return s;
  set_gr_work(net);
  cudaStream_t st = net->ctx->stream;
  const int64_t W = net->total_w, L = prm->max_block_weight;
  const int32_t max_it = prm->max_iterations > 0 ? prm->max_iterations : net->d.n_nodes + 1;
  hfp_fc_result r{};
  int32_t np = 0, it = 0;
  hfp_status status = HFP_OK;
  auto record = [&](int32_t side, int32_t node) {
    if (pierce_side && np < pierce_cap) pierce_side[np] = side;
    if (pierce_node && np < pierce_cap) pierce_node[np] = node;
    np++;
  };
  // bulk piercing bookkeeping per side (0 = S, 1 = T), as in the header
  const int64_t beta = prm->bulk_beta_pct;
  int64_t base[2] = {0, 0}, carry[2] = {0, 0}, added_w[2] = {0, 0}, added_n[2] = {0, 0};
  int64_t pre_w[2] = {0, 0};
  int32_t grown[2] = {0, 0};
  bool pending[2] = {false, false};
  if (beta > 0) {
    int64_t ws = 0, wt = 0;
    if ((s = node_weight(net, 0, &ws)) != HFP_OK) return s;
    if ((s = node_weight(net, 1, &wt)) != HFP_OK) return s;
    base[0] = beta * (W - 2 * ws) / 200;
    base[1] = beta * (W - 2 * wt) / 200;
  }
  if ((s = ensure_max_flow(net)) != HFP_OK) return s;
  it = 1;
  for (;;) {
    if ((s = ensure_source_side(net)) != HFP_OK) return s;
    Ctl c;
    if ((s = read_ctl(net, &c)) != HFP_OK) return s;
    r.flow = (int64_t)c.flow;
    if (prm->flow_bound >= 0 && (int64_t)c.flow > prm->flow_bound) {
      status = fail(HFP_ABORTED_WORSE, "flow %lld exceeds bound %lld", (long long)c.flow,
                    (long long)prm->flow_bound);
      break;
    }
    const int64_t wS = c.wS, wT = c.wT;
    for (int x = 0; x < 2; x++)
      if (pending[x]) {
        const int64_t grew = (x == 0 ? wS : wT) - pre_w[x];
        const int64_t goal = base[x] + carry[x];
        added_w[x] += grew;
        carry[x] = goal - grew > 0 ? goal - grew : 0;
        base[x] = base[x] * beta / 100;
        grown[x]++;
        pending[x] = false;
      }
    const bool balS = wS <= L && W - wS <= L;
    const bool balT = wT <= L && W - wT <= L;
    if (balS || balT) {
      bool use_t;
      if (balS && balT) {
        int64_t mS = wS > W - wS ? wS : W - wS;
        int64_t mT = wT > W - wT ? wT : W - wT;
        use_t = mT < mS;
      } else {
        use_t = !balS;
      }
      r.result_side = use_t ? 1 : 0;
      r.source_weight = use_t ? W - wT : wS;
      DevBuf best;
      if (net->n_region > 0) {
        CK(best.alloc(net->n_region, st));
        launch_region_side(net->d, use_t ? 1 : 0, net->n_region, best.as<uint8_t>(),
                           net->ctx->sms, st);
      }
      if (prm->mb_reps > 0) {
        // most balanced cut: path-free piercings from this state, mb_reps times
        NetSnapshot snap;
        if ((s = snap.take(net)) != HFP_OK) return s;
        int64_t best_max = r.source_weight > W - r.source_weight ? r.source_weight
                                                                  : W - r.source_weight;
        for (int32_t rep = 0; rep < prm->mb_reps; rep++) {
          if (rep > 0 && (s = snap.restore(net)) != HFP_OK) return s;
          const uint32_t seed = prm->seed + (uint32_t)rep;
          for (;;) {
            if ((s = ensure_source_side(net)) != HFP_OK) return s;
            Ctl cm;
            if ((s = read_ctl(net, &cm)) != HFP_OK) return s;
            for (int ut = 0; ut < 2; ut++) {
              const int64_t w0 = ut ? W - cm.wT : cm.wS;
              if (w0 > L || W - w0 > L) continue;
              const int64_t mx = w0 > W - w0 ? w0 : W - w0;
              if (mx < best_max) {
                best_max = mx;
                r.source_weight = w0;
                r.result_side = 2;
                if (net->n_region > 0)
                  launch_region_side(net->d, ut, net->n_region, best.as<uint8_t>(),
                                     net->ctx->sms, st);
              }
            }
            const int grow_s = cm.wS <= cm.wT;
            int32_t p = -1;
            bool no_path = false;
            s = select_pierce(net, grow_s, prm, &p, &no_path, -1, 0, nullptr, seed, true);
            if (s == HFP_NO_BALANCED_CUT) break;
            if (s != HFP_OK) return s;
            if (!no_path) break;   // only piercings that open no augmenting path
            record(grow_s ? 2 : 3, p);
            r.mb_steps++;
            if ((s = pierce(net, grow_s ? 0 : 1, &p, 1, true)) != HFP_OK) return s;
          }
        }
        set_last_error("");
      }
      if (final_side && net->n_region > 0) {
        CK(cudaMemcpyAsync(final_side, best.p, net->n_region, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
      }
      break;
    }
    if (it >= max_it) {
      status = fail(HFP_ERR_ITER_LIMIT, "FlowCutter iteration limit %d reached", max_it);
      break;
    }
    const int grow_s = wS <= wT;
    const int x = grow_s ? 0 : 1;
    const int64_t wR = grow_s ? wS : wT;
    int32_t p = -1;
    bool no_path = false;
    unsigned long long key = 0;
    if ((s = select_pierce(net, grow_s, prm, &p, &no_path, -1, 0, &key)) != HFP_OK) {
      status = s;
      break;
    }
    // bulk piercing: how many nodes this iteration takes
    int64_t k = 1;
    if (beta > 0) {
      const int64_t goal = base[x] + carry[x];
      const bool far = 2 * (wR + goal) <= W;
      if (!no_path && far && grown[x] >= prm->bulk_warmup && added_n[x] > 0) {
        int64_t avg = added_w[x] / added_n[x];
        if (avg < 1) avg = 1;
        k = (goal + avg - 1) / avg;
        if (k < 1) k = 1;
      }
    }
    std::vector<int32_t> nodes{p};
    if (k > 1) {
      int64_t taken_w = 0;
      if ((s = node_weight(net, p, &taken_w)) != HFP_OK) return s;
      while ((int64_t)nodes.size() < k) {
        int32_t q = -1;
        unsigned long long kq = 0;
        s = select_pierce(net, grow_s, prm, &q, nullptr, wR + taken_w, key, &kq);
        if (s == HFP_NO_BALANCED_CUT) break;
        if (s != HFP_OK) return s;
        int64_t wq = 0;
        if ((s = node_weight(net, q, &wq)) != HFP_OK) return s;
        nodes.push_back(q);
        taken_w += wq;
        key = kq;
      }
      set_last_error("");
      if (nodes.size() > 1) r.bulk_steps++;
    }
    for (int32_t q : nodes) record(x, q);
    pre_w[x] = wR;
    added_n[x] += (int64_t)nodes.size();
    pending[x] = true;
    if ((s = pierce(net, x, nodes.data(), (int32_t)nodes.size(),
                    nodes.size() == 1 && no_path)) != HFP_OK)
      return s;
    it++;
  }
  r.iterations = it;
  r.n_pierced = np;
  if (result) *result = r;
  if (status == HFP_OK && (pierce_side || pierce_node) && np > pierce_cap)
    status = fail(HFP_ERR_BUFFER_TOO_SMALL, "piercing sequence has %d entries", np);
  return status;
}
