// Batched FlowCutter: many flow networks in one launch of fc_batch_kernel
// (engine_batch.cuh), with a device work queue handing the networks to groups
// of CTAs.  Groups of up to kMaxClusterCtas CTAs are thread-block clusters
// (barriers in distributed shared memory); larger groups share a cooperative
// launch.  Used by hfp_flowcutter_batch and by the batched k-way round
// (kway.cu).
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "internal.h"

using namespace hfp;

namespace hfp {

// CTAs per SM of fc_batch_kernel at kEngineThreads threads (at most 2).
hfp_status batch_grid(hfp_ctx* ctx, int* grid) {
  static int per_sm_cache[64] = {0};
  int dev = ctx->device;
  int per_sm = dev < 64 ? per_sm_cache[dev] : 0;
  if (per_sm == 0) {
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fc_batch_kernel, kEngineThreads,
                                                     0));
    if (per_sm < 1) return fail(HFP_ERR_CUDA, "fc_batch_kernel cannot be resident");
    if (per_sm > 2) per_sm = 2;
    if (dev < 64) per_sm_cache[dev] = per_sm;
  }
  *grid = ctx->sms * per_sm;
  return HFP_OK;
}

hfp_status run_fc_batch(hfp_ctx* ctx, BatchItem* items, int n, int group_ctas, float* ms_out,
                        const BatchTune* tune) {
  if (n == 0) return HFP_OK;
  cudaStream_t st = ctx->stream;
  int grid = 0;
  hfp_status s = batch_grid(ctx, &grid);
  if (s != HFP_OK) return s;
  int G = group_ctas;
  if (G <= 0) {
    // one group per job when the grid allows, else as many as fit
    G = grid / n;
    if (G < 1) G = 1;
  }
  if (G > grid) G = grid;
  // big groups first (the largest jobs start on them), then groups of G
  int Gb = (int)ctx->batch_big_ctas, big = (int)ctx->batch_big_groups;
  if (Gb <= G || big <= 0) {
    Gb = G;
    big = 0;
  }
  if (big > n) big = n;
  while (big > 0 && big * Gb > grid) big--;
  int groups = big + (grid - big * Gb) / G;
  bool cluster = big == 0 && ctx->batch_cluster && G <= kMaxClusterCtas;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  if (cluster) {
    // clusters when as many of them can be resident as there are groups; with
    // batch_cluster = 2 the launch has only as many groups as can be resident
    // clusters (fewer groups, every barrier in distributed shared memory)
    CK(cudaFuncSetAttribute(fc_batch_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    cfg.gridDim = dim3(groups * G);
    cfg.blockDim = dim3(kEngineThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = G;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int resident = 0;
    CK(cudaOccupancyMaxActiveClusters(&resident, fc_batch_kernel, &cfg));
    if (resident < groups && ctx->batch_cluster == 2 && resident >= 1) {
      groups = resident;
      cfg.gridDim = dim3(groups * G);
    }
    cluster = resident >= groups;
  }
  ctx->last_groups = groups;
  ctx->last_group_ctas = G;
  ctx->last_cluster = cluster ? 1 : 0;
  if (groups > kMaxGroups) return fail(HFP_ERR_INVALID, "too many groups");
  const int launch = big * Gb + (groups - big) * G;
  if (launch > kMaxBatchCtas) return fail(HFP_ERR_INVALID, "grid above %d CTAs", kMaxBatchCtas);
  // jobs, largest network first
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    return items[a].net->d.p_pins > items[b].net->d.p_pins;
  });
  Params P0 = ctx->params;
  P0.fused_rounds = ctx->batch_fused_rounds;
  P0.async_gr = ctx->batch_async_gr;
  P0.stall_rounds_pierce = ctx->batch_stall_rounds_pierce;
  uint32_t gr_work_x100 = ctx->batch_gr_work_x100;
  if (tune) {   // the tuned speed knobs; budgets and wait bounds stay the context's
    P0 = tune->P;
    P0.max_rounds = ctx->params.max_rounds;
    P0.timeout_ns = ctx->params.timeout_ns;
    gr_work_x100 = tune->gr_work_x100;
  }
  std::vector<FcJob> jobs(n);
  for (int t = 0; t < n; t++) {
    BatchItem& it = items[order[t]];
    hfp_net* net = it.net;
    if (net->flow_started) return fail(HFP_ERR_STATE, "batched FlowCutter needs fresh networks");
    if (it.params.bulk_beta_pct || it.params.mb_reps)
      return fail(HFP_ERR_INVALID,
                  "bulk piercing and the most balanced cut are not supported in the batched launch");
    // a network without these buffers runs two-phase rounds and level-by-level
    // relabels (the kernel checks per job)
    if (hfp_status s2 = ensure_engine_buffers(net, P0)) return s2;
    if (!net->d.net_done) {
      const size_t mb = net->d.m_nets > 0 ? (size_t)net->d.m_nets : 1;
      CK(cudaMallocAsync(&net->net_done_buf, mb, st));
      CK(cudaMemsetAsync(net->net_done_buf, 0, mb, st));
      net->d.net_done = (uint8_t*)net->net_done_buf;
    }
    FcJob& J = jobs[t];
    memset(&J, 0, sizeof(J));
    J.N = net->d;
    J.E = net->E;
    J.total_w = net->total_w;
    J.max_w = it.params.max_block_weight;
    J.flow_bound = it.params.flow_bound;
    J.gr_work = (unsigned long long)net->d.NL * gr_work_x100 / 100 + 1024;
    J.pierce_node = it.pierce_node_dev;
    J.pierce_side = it.pierce_side_dev;
    J.pierce_cap = it.pierce_cap;
    J.seed = it.params.seed;
    J.max_it = it.params.max_iterations > 0 ? it.params.max_iterations : net->d.n_nodes + 1;
    J.dist_ready = net->dist_ready ? 1 : 0;
    launch_engine_setup(net->E, SETUP_BATCH, st);
  }
  DevBuf djobs, dctl;
  CK(djobs.alloc(sizeof(FcJob) * n, st));
  CK(dctl.alloc(sizeof(BatchCtl), st));
  CK(cudaMemcpyAsync(djobs.p, jobs.data(), sizeof(FcJob) * n, cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(dctl.p, 0, sizeof(BatchCtl), st));
  FcJob* jp = djobs.as<FcJob>();
  BatchCtl* bp = dctl.as<BatchCtl>();
  int use_cluster = cluster ? 1 : 0;
  void* args[] = {(void*)&jp,     (void*)&n,      (void*)&bp, (void*)&G,          (void*)&Gb,
                  (void*)&big,    (void*)&groups, (void*)&P0, (void*)&use_cluster};
  CK(cudaEventRecord(ctx->ev0, st));
  if (cluster)
    CK(cudaLaunchKernelEx(&cfg, fc_batch_kernel, jp, n, bp, G, Gb, big, groups, P0, use_cluster));
  else
    CK(cudaLaunchCooperativeKernel((void*)fc_batch_kernel, dim3(launch), dim3(kEngineThreads),
                                   args, 0, st));
  CK(cudaEventRecord(ctx->ev1, st));
  count_launches(1);
  int berr = 0;
  CK(cudaMemcpyAsync(jobs.data(), djobs.p, sizeof(FcJob) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&berr, &bp->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  if (ms_out) *ms_out = ms;
  if (berr) return fail(HFP_ERR_CUDA, "batched FlowCutter: a group barrier timed out");
  hfp_status first_err = HFP_OK;
  for (int t = 0; t < n; t++) {
    BatchItem& it = items[order[t]];
    const FcJob& J = jobs[t];
    for (int k = 0; k < kStateSlots; k++) {
      ctx->batch_ns[k] += J.st_ns[k];
      ctx->batch_cnt[k] += J.st_cnt[k];
      ctx->batch_lin[k] += J.st_lin[k];
      ctx->batch_hin[k] += J.st_hin[k];
    }
    hfp_net* net = it.net;
    net->flow_started = true;
    net->launches++;
    it.result.flow = J.flow;
    it.result.source_weight = J.source_weight;
    it.result.iterations = J.iterations;
    it.result.n_pierced = J.n_pierced;
    it.result.result_side = J.result_side;
    it.result.device_us = (int32_t)std::min<unsigned long long>(J.device_ns / 1000, 0x7fffffffull);
    it.group_ctas = J.group_ctas;
    if (J.status >= 100) {
      it.status = J.status - 100 == kDevBadInput ? HFP_ERR_INVALID : HFP_ERR_ITER_LIMIT;
      if (first_err == HFP_OK)
        first_err = fail(it.status, "batched FlowCutter: device code %d", J.status - 100);
      continue;
    }
    it.status = J.status;
    net->labels_exact = true;
    net->sr_valid = true;
  }
  return first_err;
}

}  // namespace hfp

HFP_API hfp_status hfp_flowcutter_batch(hfp_ctx* ctx, hfp_fc_task* tasks, int32_t n,
                                        int32_t group_ctas) {
  if (!ctx || n < 0 || (n > 0 && !tasks)) return fail(HFP_ERR_INVALID, "bad arguments");
  if (n == 0) return HFP_OK;
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  std::vector<BatchItem> items(n);
  std::vector<DevBuf> pn(n), ps(n);
  for (int i = 0; i < n; i++) {
    hfp_fc_task& t = tasks[i];
    if (!t.net || t.net->ctx != ctx) return fail(HFP_ERR_INVALID, "task %d: bad network", i);
    if (t.pierce_cap < 0) return fail(HFP_ERR_INVALID, "task %d: negative pierce_cap", i);
    for (int j = 0; j < i; j++)
      if (tasks[j].net == t.net) return fail(HFP_ERR_INVALID, "task %d repeats a network", i);
    items[i].net = t.net;
    items[i].params = t.params;
    items[i].pierce_cap = (t.pierce_side || t.pierce_node) ? t.pierce_cap : 0;
    if (items[i].pierce_cap > 0) {
      CK(pn[i].alloc(sizeof(int32_t) * items[i].pierce_cap, st));
      CK(ps[i].alloc(items[i].pierce_cap, st));
      items[i].pierce_node_dev = pn[i].as<int32_t>();
      items[i].pierce_side_dev = ps[i].as<int8_t>();
    }
  }
  hfp_status s = run_fc_batch(ctx, items.data(), n, group_ctas, nullptr);
  if (s != HFP_OK) return s;
  hfp_status ret = HFP_OK;
  for (int i = 0; i < n; i++) {
    hfp_fc_task& t = tasks[i];
    BatchItem& it = items[i];
    t.result = it.result;
    t.status = it.status;
    const int k = std::min(it.result.n_pierced, it.pierce_cap);
    if (k > 0) {
      std::vector<int8_t> side(k);
      if (t.pierce_node)
        CK(cudaMemcpyAsync(t.pierce_node, pn[i].p, sizeof(int32_t) * k, cudaMemcpyDeviceToHost,
                           st));
      CK(cudaMemcpyAsync(side.data(), ps[i].p, k, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (t.pierce_side)
        for (int j = 0; j < k; j++) t.pierce_side[j] = side[j];
    }
    if (it.status == HFP_OK && t.final_side && t.net->n_region > 0) {
      DevBuf tmp;
      CK(tmp.alloc(t.net->n_region, st));
      launch_region_side(t.net->d, it.result.result_side, t.net->n_region, tmp.as<uint8_t>(),
                         ctx->sms, st);
      CK(cudaMemcpyAsync(t.final_side, tmp.p, t.net->n_region, cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
    }
    if (it.status == HFP_OK && (t.pierce_side || t.pierce_node) &&
        it.result.n_pierced > t.pierce_cap && ret == HFP_OK)
      ret = fail(HFP_ERR_BUFFER_TOO_SMALL, "task %d: piercing sequence has %d entries", i,
                 it.result.n_pierced);
  }
  return ret;
}

HFP_API hfp_status hfp_ctx_batch_profile(hfp_ctx* ctx, uint64_t* state_ns, uint64_t* state_cnt,
                                         uint64_t* light_in, uint64_t* heavy_in,
                                         int32_t n_states, int32_t reset) {
  if (!ctx || n_states < 0) return fail(HFP_ERR_INVALID, "bad arguments");
  const int k = std::min<int>(n_states, kStateSlots);
  for (int i = 0; i < k; i++) {
    if (state_ns) state_ns[i] = ctx->batch_ns[i];
    if (state_cnt) state_cnt[i] = ctx->batch_cnt[i];
    if (light_in) light_in[i] = ctx->batch_lin[i];
    if (heavy_in) heavy_in[i] = ctx->batch_hin[i];
  }
  if (reset) {
    for (int i = 0; i < kStateSlots; i++)
      ctx->batch_ns[i] = ctx->batch_cnt[i] = ctx->batch_lin[i] = ctx->batch_hin[i] = 0;
  }
  return HFP_OK;
}

HFP_API hfp_status hfp_ctx_last_batch_layout(hfp_ctx* ctx, int32_t* groups, int32_t* group_ctas,
                                            int32_t* cluster) {
  if (!ctx) return fail(HFP_ERR_INVALID, "ctx is NULL");
  if (groups) *groups = ctx->last_groups;
  if (group_ctas) *group_ctas = ctx->last_group_ctas;
  if (cluster) *cluster = ctx->last_cluster;
  return HFP_OK;
}

HFP_API hfp_status hfp_ctx_wait_selftest(hfp_ctx* ctx, int32_t barrier, float* waited_ms) {
  if (!ctx || barrier < 0 || barrier > 2) return fail(HFP_ERR_INVALID, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t st = ctx->stream;
  DevBuf e, b;
  CK(e.alloc(sizeof(EngineCtl), st));
  CK(b.alloc(sizeof(BatchCtl), st));
  CK(cudaMemsetAsync(e.p, 0, sizeof(EngineCtl), st));
  CK(cudaMemsetAsync(b.p, 0, sizeof(BatchCtl), st));
  EngineCtl* E = e.as<EngineCtl>();
  BatchCtl* B = b.as<BatchCtl>();
  const unsigned long long tns = ctx->params.timeout_ns;
  const int ctas = 2, threads = 128;
  CK(cudaEventRecord(ctx->ev0, st));
  if (barrier == 2) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    cfg.gridDim = dim3(ctas);
    cfg.blockDim = dim3(threads);
    cfg.stream = st;
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ctas;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK(cudaLaunchKernelEx(&cfg, wait_selftest_kernel, E, B, (int)barrier, tns));
  } else {
    wait_selftest_kernel<<<ctas, threads, 0, st>>>(E, B, barrier, tns);
    CK(cudaGetLastError());
  }
  CK(cudaEventRecord(ctx->ev1, st));
  count_launches(1);
  int err = 0;
  CK(cudaMemcpyAsync(&err, barrier == 0 ? &E->c.err : &B->err, sizeof(int),
                     cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  if (waited_ms) *waited_ms = ms;
  if (err != 0) return fail(HFP_ERR_ITER_LIMIT, "device wait ran out after %.1f ms", ms);
  return HFP_OK;
}
