// Allocation-free maximum flow and minimal source-side cut.
//
// Some callers cannot allocate device memory at the point where they need a
// flow: a plug-in that must stay within a host application's fixed
// device-memory budget or custom allocator, or a latency-critical loop in
// which allocation is not allowed (cudaMalloc can synchronise the device or
// fail under memory pressure).  hfp_max_flow_noalloc serves them: it runs
// the same engine kernel as hfp_max_flow / hfp_min_cut_source_side, but all
// of its working state lives in one file-scope __device__ array of fixed
// size, so the call itself never allocates or frees memory.  The caller
// passes the flow network (in the layout hfp_net_export writes) and the
// output buffers.  The call synchronises its stream and reads two status
// words back to the host, so it cannot be recorded into a CUDA graph.
//
// The array is part of the library image: every GPU that loads the library
// holds it until the process exits.  Each call clears the part it uses.
// Calls that overlap on the GPU (for example on two streams) share the array
// and race; serialise them.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "hfp.h"
#include "kernels.cuh"

namespace hfp {

constexpr size_t kStaticScratchBytes = size_t(24) << 20;   // 24 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

// Per-device set-up: the device address of g_static_scratch (host code may
// only use the symbol through cudaGetSymbolAddress) and the cooperative
// grid size of the engine kernel.
struct StaticDevice {
  bool ready = false;
  unsigned char* scratch = nullptr;
  int coop_grid = 0;
};
constexpr int kMaxDevices = 64;
StaticDevice g_static_dev[kMaxDevices];
std::mutex g_static_mu;

inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Bytes of g_static_scratch a network needs (the carving in hfp_max_flow_noalloc).
size_t static_bytes(int64_t NL, int64_t m, int64_t p) {
  size_t b = align256(sizeof(EngineCtl)) + align256(64);
  b += 2 * align256(sizeof(int32_t) * NL);                       // labels
  b += 2 * align256(sizeof(long long) * NL);                     // excess, delta
  b += align256(sizeof(uint32_t) * NL);                          // stamps
  b += 3 * align256((size_t)NL);                                 // flags, needrl, insr
  b += 4 * align256(sizeof(int32_t) * NL);                       // lists
  b += 2 * align256(sizeof(int32_t) * p) + align256(sizeof(int32_t) * m);  // flows
  b += align256(sizeof(int2) * p) + align256(sizeof(int32_t) * p);        // inc, slot_net
  return b;
}

}  // namespace

// Bounds and consistency of the caller's network; err[0] = 1 on any
// violation.  Every incidence entry of hypernode u must name a pin slot
// holding u, and every slot must be named once (mark[] counts, zeroed by the
// caller; k_static_check_marks reads them).  Offsets are validated before
// they index anything.
__global__ void k_static_check(int32_t n, int32_t m, long long p, const uint32_t* net_off,
                               const int32_t* pins, const int32_t* net_w, const uint32_t* node_off,
                               const int32_t* inc_slot, const int32_t* node_w, int* mark,
                               int* err) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long nth = (long long)gridDim.x * blockDim.x;
  if (tid == 0 && (net_off[0] != 0 || (long long)net_off[m] != p || node_off[0] != 0 ||
                   (long long)node_off[n] != p))
    err[0] = 1;
  for (long long e = tid; e < m; e += nth)
    if (net_off[e + 1] < net_off[e] || (long long)net_off[e + 1] > p || net_w[e] <= 0) err[0] = 1;
  for (long long j = tid; j < p; j += nth) {
    const int v = pins[j];
    const int s = inc_slot[j];
    if (v < 0 || v >= n || s < 0 || (long long)s >= p) err[0] = 1;
  }
  for (long long u = tid; u < n; u += nth) {
    const uint32_t b = node_off[u], e = node_off[u + 1];
    if (e < b || (long long)e > p || node_w[u] < 0) {
      err[0] = 1;
      continue;
    }
    for (uint32_t j = b; j < e; j++) {
      const int s = inc_slot[j];
      if (s < 0 || (long long)s >= p) continue;   // reported above
      if (pins[s] != (int)u) err[0] = 1;
      atomicAdd(&mark[s], 1);
    }
  }
}

// every pin slot named by exactly one incidence entry
__global__ void k_static_check_marks(long long p, const int* mark, int* err) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p;
       j += (long long)gridDim.x * blockDim.x)
    if (mark[j] != 1) err[0] = 1;
}

// slot -> net of the caller's net CSR, warp per net
__global__ void k_static_slot_net(int32_t m, const uint32_t* net_off, int32_t* slot_net) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw)
    for (unsigned p = net_off[e] + lane; p < net_off[e + 1]; p += 32) slot_net[p] = (int32_t)e;
}

// (net, slot) pairs of the hypernode incidence lists
__global__ void k_static_inc(long long p, const int32_t* inc_slot, const int32_t* slot_net,
                             int2* inc) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < p;
       j += (long long)gridDim.x * blockDim.x) {
    const int s = inc_slot[j];
    inc[j] = make_int2(slot_net[s], s);
  }
}

// terminals and engine control of a fresh flow problem ({s}, {t})
__global__ void k_static_init(NetDev N, EngineCtl* E) {
  N.flags[0] = kSource;
  N.flags[1] = kSink;
  E->s.epoch = 1;
  E->s.state = ST_DONE;
}

}  // namespace hfp

using namespace hfp;

namespace hfp {
void set_last_error(const char* msg);
}

static hfp_status noalloc_fail(hfp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define CKS(call)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return noalloc_fail(HFP_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));   \
  } while (0)

extern "C" __attribute__((visibility("default"))) hfp_status hfp_max_flow_noalloc(
    int device, void* stream, const hfp_flow_network_view* v, int64_t* flow_value,
    uint8_t* in_source_lawler, int64_t* source_weight) {
  if (!v) return noalloc_fail(HFP_ERR_INVALID, "network view is NULL");
  if (device < 0 || device >= kMaxDevices) return noalloc_fail(HFP_ERR_INVALID, "bad device %d", device);
  const int64_t n = v->n_nodes, m = v->m_nets, p = v->p_pins;
  if (n < 2 || m < 0 || p < 0 || p >= (1ll << 31))
    return noalloc_fail(HFP_ERR_INVALID, "bad network sizes n=%lld m=%lld p=%lld", (long long)n,
                        (long long)m, (long long)p);
  const int64_t NL = n + 2 * m;
  const size_t need = static_bytes(NL, m, p);
  if (NL >= (1ll << 31) - 2 || need > kStaticScratchBytes)
    return noalloc_fail(HFP_ERR_INVALID,
                        "network needs %zu bytes of static scratch; the maximum is %zu "
                        "(use hfp_build_flow_network / hfp_max_flow instead)",
                        need, kStaticScratchBytes);
  if (!v->net_off || !v->node_off || !v->node_w || (p > 0 && (!v->pins || !v->inc_slot)) ||
      (m > 0 && !v->net_w))
    return noalloc_fail(HFP_ERR_INVALID, "missing network array");
  CKS(cudaSetDevice(device));
  cudaStream_t st = (cudaStream_t)stream;

  // once per device, with the device current: scratch address, grid size
  StaticDevice dev;
  {
    std::lock_guard<std::mutex> lk(g_static_mu);
    StaticDevice& sd = g_static_dev[device];
    if (!sd.ready) {
      void* ptr = nullptr;
      CKS(cudaGetSymbolAddress(&ptr, g_static_scratch));
      int sms = 0, per_sm = 0;
      CKS(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
      CKS(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, engine_kernel, kEngineThreads, 0));
      if (per_sm < 1) return noalloc_fail(HFP_ERR_CUDA, "engine kernel does not fit on an SM");
      sd.scratch = (unsigned char*)ptr;
      sd.coop_grid = sms * (per_sm > 2 ? 2 : per_sm);
      sd.ready = true;
    }
    dev = sd;
  }

  // carve the working state out of the static array (layout of static_bytes)
  unsigned char* q = dev.scratch;
  auto take = [&](size_t bytes) {
    unsigned char* r = q;
    q += align256(bytes);
    return r;
  };
  EngineCtl* E = (EngineCtl*)take(sizeof(EngineCtl));
  int* misc = (int*)take(64);            // [0] input check flag, [1] saturated node id (0 = s)
  NetDev D{};
  D.n_nodes = (int32_t)n;
  D.m_nets = (int32_t)m;
  D.NL = (int32_t)NL;
  D.p_pins = p;
  D.lab0 = (int32_t*)take(sizeof(int32_t) * NL);
  D.lab1 = (int32_t*)take(sizeof(int32_t) * NL);
  D.excess = (long long*)take(sizeof(long long) * NL);
  D.delta = (long long*)take(sizeof(long long) * NL);
  D.stamp = (uint32_t*)take(sizeof(uint32_t) * NL);
  D.flags = (uint8_t*)take((size_t)NL);
  D.needrl = (uint8_t*)take((size_t)NL);
  D.insr = (uint8_t*)take((size_t)NL);
  for (int k = 0; k < 4; k++) D.list[k] = (int32_t*)take(sizeof(int32_t) * NL);
  D.f_in = (int32_t*)take(sizeof(int32_t) * p);
  D.f_out = (int32_t*)take(sizeof(int32_t) * p);
  D.f_b = (int32_t*)take(sizeof(int32_t) * m);
  int2* inc = (int2*)take(sizeof(int2) * p);
  int32_t* slot_net = (int32_t*)take(sizeof(int32_t) * p);
  const size_t used = (size_t)(q - dev.scratch);
  D.net_off = v->net_off;
  D.pin = v->pins;
  D.net_w = v->net_w;
  D.node_off = v->node_off;
  D.inc = inc;
  D.node_w = v->node_w;
  D.node_dist = nullptr;   // not read by max flow / source-side cut
  D.node_orig = nullptr;
  D.node_gid = nullptr;

  // the array keeps the previous call's contents: clear everything used
  CKS(cudaMemsetAsync(dev.scratch, 0, used, st));
  // slot_net doubles as the slot marks of the check (zeroed above, refilled below)
  k_static_check<<<256, 256, 0, st>>>(D.n_nodes, D.m_nets, p, v->net_off, v->pins, v->net_w,
                                      v->node_off, v->inc_slot, v->node_w, slot_net, misc);
  k_static_check_marks<<<256, 256, 0, st>>>(p, slot_net, misc);
  count_launches(2);
  int herr = 0;
  CKS(cudaMemcpyAsync(&herr, misc, sizeof(int), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (herr) return noalloc_fail(HFP_ERR_INVALID, "network arrays out of bounds or malformed");

  if (m > 0) {
    k_static_slot_net<<<(unsigned)((m * 32 + 255) / 256 < 4096 ? (m * 32 + 255) / 256 : 4096), 256,
                        0, st>>>(D.m_nets, v->net_off, slot_net);
    count_launches(1);
  }
  if (p > 0) {
    k_static_inc<<<(unsigned)((p + 255) / 256 < 4096 ? (p + 255) / 256 : 4096), 256, 0, st>>>(
        p, v->inc_slot, slot_net, inc);
    count_launches(1);
  }
  k_static_init<<<1, 1, 0, st>>>(D, E);
  count_launches(1);
  launch_heavy_flags(D, dev.coop_grid / 2 > 0 ? dev.coop_grid / 2 : 1, st);

  Params P{};
  P.timeout_ns = 10ull * 1000 * 1000 * 1000;
  P.max_rounds = 1ull << 22;
  P.gr_work = 2ull * (unsigned long long)NL + 1024;
  P.stall_rounds = 200;
  P.stall_nodes = 1500;
  P.tail_enter = 64;
  P.tail_exit = 192;
  P.bfs_enter = 0;
  P.bfs_exit = 0;
  P.pierce_relabel = 0;
  P.stall_rounds_pierce = 0;
  P.stall_adapt = 0;
  void* args[] = {(void*)&D, (void*)&E, (void*)&P};

  // maximum preflow from {s} to {t}: saturate s, global relabel, rounds
  launch_engine_setup(E, SETUP_PREP, st);
  launch_saturate(D, E, misc + 1, 1, st);
  launch_engine_setup(E, SETUP_GR, st);
  CKS(cudaLaunchCooperativeKernel((void*)engine_kernel, dim3(dev.coop_grid), dim3(kEngineThreads),
                                  args, 0, st));
  count_launches(1);
  Ctl c;
  CKS(cudaMemcpyAsync(&c, &E->c, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  CKS(cudaStreamSynchronize(st));
  if (c.err != kDevOk)
    return noalloc_fail(c.err == kDevBadInput ? HFP_ERR_INVALID : HFP_ERR_ITER_LIMIT,
                        "flow engine stopped: device code %d", c.err);
  // minimal source side S_r
  launch_engine_setup(E, SETUP_SR, st);
  CKS(cudaLaunchCooperativeKernel((void*)engine_kernel, dim3(dev.coop_grid), dim3(kEngineThreads),
                                  args, 0, st));
  count_launches(1);
  CKS(cudaMemcpyAsync(&c, &E->c, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  if (in_source_lawler)
    CKS(cudaMemcpyAsync(in_source_lawler, D.insr, (size_t)NL, cudaMemcpyDeviceToDevice, st));
  CKS(cudaStreamSynchronize(st));
  if (c.err != kDevOk)
    return noalloc_fail(c.err == kDevBadInput ? HFP_ERR_INVALID : HFP_ERR_ITER_LIMIT,
                        "flow engine stopped: device code %d", c.err);
  if (flow_value) *flow_value = (int64_t)c.flow;
  if (source_weight) *source_weight = c.wS;
  return HFP_OK;
}
