// Host-side launchers of the device kernels, shared by the translation units.
#pragma once
#include "engine.cuh"

namespace hfp {

constexpr int32_t kDistFar = (1 << 20) - 1;

// launches of this library's kernels (process-wide, host side)
void count_launches(unsigned k);
unsigned long long launches_total();

// build.cu
size_t scan_scratch_words(unsigned n);
void scan_exclusive(unsigned* a, unsigned n, unsigned* scratch, unsigned* total, cudaStream_t st);
void launch_region_map(int32_t n, int32_t n_region, const int32_t* region, const int32_t* side,
                       const int32_t* node_w_h, int32_t* loc, int32_t* node_gid, int32_t* node_w,
                       int8_t* node_orig, int* err, cudaStream_t st);
// verts / nets (may be null): the vertices / ascending nets to scan (n / m
// is then their count); per-net outputs are indexed by list position
void launch_st_weight(int32_t n, const int32_t* verts, const int32_t* loc, const int32_t* side,
                      const int32_t* node_w_h, unsigned long long* wsum, int* err, int sms,
                      cudaStream_t st);
void launch_net_scan(int32_t n, int32_t m, const int32_t* nets, const uint32_t* net_off,
                     const int32_t* pins, const int32_t* net_w, const int32_t* side,
                     const int32_t* loc, unsigned* keep, unsigned* size, unsigned* has_s,
                     unsigned* has_t, int32_t* dist_tmp, int mark_dist, unsigned long long* wnet,
                     int* err, int sms, cudaStream_t st);
void launch_net_fill(int32_t m, const int32_t* nets, const uint32_t* net_off,
                     const int32_t* pins, const int32_t* net_w, const int32_t* loc,
                     const unsigned* keep,
                     const unsigned* net_pos, const unsigned* pin_pos, const unsigned* s_pos,
                     const unsigned* t_pos, const unsigned* has_s, const unsigned* has_t,
                     const unsigned* totals, uint32_t* nnet_off, int32_t* npin, int32_t* nnet_w,
                     int32_t* nnet_gid, int2* inc, int sms, cudaStream_t st);
void launch_incidence(int32_t n_nodes, int32_t m_net, unsigned p, const uint32_t* nnet_off,
                      const int32_t* npin, unsigned* deg_then_off, unsigned* cursor,
                      const unsigned* totals, int2* inc, int2* tmp, unsigned* scan_scratch,
                      unsigned* scan_total, int sms, cudaStream_t st);
void launch_dist_seed(int32_t n_nodes, const int32_t* dist_tmp, int32_t* dist, int sms,
                      cudaStream_t st);
void launch_heavy_flags(const NetDev& N, int sms, cudaStream_t st);
void launch_dist_export(int32_t n_nodes, const int32_t* dist, int32_t* out, int sms,
                        cudaStream_t st);
void launch_dist_copy(int32_t n_region, const int32_t* dist_in, int32_t* dist, int* err,
                      cudaStream_t st);
void launch_st_attrs(int32_t* node_gid, int32_t* node_w, int8_t* node_orig,
                     const unsigned long long* wsum, uint8_t* flags, int* err, cudaStream_t st);
// Second construction algorithm (Section 6).  sort_build_count: the number
// of (net, vertex) pairs of the region (deg[nr] becomes their offsets);
// synchronises.  sort_build_runs: the pairs sorted by net (stable) as runs
// run_start[R + 1] / run_net[R] over key / val (key2 / val2: second buffers;
// head, rid: scratch of the pair count; hist: 256 counters per tile of 512
// pairs); synchronises.  Then per run the first algorithm's keep / size /
// s / t rules from the pins of blocks b0 / b1 in H (cnt[noff[e] + rank of the
// block in mask[e]]), and the fill of the kept nets.
cudaError_t sort_build_count(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                             unsigned* deg, unsigned* scr, unsigned* tot, unsigned* n_pairs,
                             int sms, cudaStream_t st);
cudaError_t sort_build_runs(int32_t nr, const int32_t* region, const uint32_t* vnet_off,
                            const int32_t* vnet, int32_t m, unsigned P2, const unsigned* pos,
                            unsigned* scr, unsigned* tot, unsigned* key, int32_t* val,
                            unsigned* key2, int32_t* val2, unsigned* hist, unsigned* head,
                            unsigned* rid, unsigned* run_start, int32_t* run_net, unsigned* R,
                            int sms, cudaStream_t st);
void launch_sb_eval(unsigned R, const unsigned* run_start, const int32_t* run_net,
                    const int32_t* val, const int32_t* region, const int32_t* side,
                    const int32_t* net_w, const unsigned long long* mask, const unsigned* noff,
                    const unsigned* cnt, int32_t b0, int32_t b1, unsigned* keep, unsigned* size,
                    unsigned* has_s, unsigned* has_t, unsigned long long* wnet, int sms,
                    cudaStream_t st);
void launch_sb_fill(unsigned R, const unsigned* run_start, const int32_t* run_net,
                    const int32_t* val, const int32_t* side, const int32_t* region,
                    const int32_t* net_w, const unsigned* keep, const unsigned* net_pos,
                    const unsigned* pin_pos, const unsigned* s_pos, const unsigned* t_pos,
                    const unsigned* has_s, const unsigned* has_t, const unsigned* totals,
                    uint32_t* nnet_off, int32_t* npin, int32_t* nnet_w, int32_t* nnet_gid,
                    int2* inc, int sms, cudaStream_t st);
// identical net removal (Section 6): group tags, smallest id per group and
// representatives; merged weights and kept-net flags / sizes / s-t
// membership; compaction; new totals; s / t incidences of the kept nets
void launch_net_tags(int32_t m, const uint32_t* off, const int32_t* pin, unsigned long long* tag,
                     unsigned long long* tab_tag, int32_t* tab_min, unsigned mask, int32_t* rep,
                     int* err, int sms, cudaStream_t st);
void launch_net_merge(int32_t m, const uint32_t* off, const int32_t* pin, const int32_t* net_w,
                      const int32_t* rep, unsigned long long* wacc, unsigned* keep,
                      unsigned* size, unsigned* has_s, unsigned* has_t, int sms, cudaStream_t st);
void launch_net_compact(int32_t m, const uint32_t* off, const int32_t* pin, const int32_t* gid,
                        const unsigned* keep, const unsigned* new_e, const unsigned* new_p,
                        const unsigned long long* wacc, uint32_t* o_off, int32_t* o_pin,
                        int32_t* o_w, int32_t* o_gid, int sms, cudaStream_t st);
void launch_dedup_totals(unsigned m_new, unsigned p_new, const unsigned* has_s_tot,
                         const unsigned* has_t_tot, uint32_t* n_off, unsigned* totals,
                         cudaStream_t st);
void launch_st_inc(int32_t m, const uint32_t* off, const unsigned* keep, const unsigned* new_e,
                   const unsigned* has_s, const unsigned* has_t, const unsigned* pos_s,
                   const unsigned* pos_t, const unsigned* node_off, const uint32_t* n_off,
                   int2* inc, int sms, cudaStream_t st);

// engine.cu
constexpr int kEngineThreads = 512;   // block scans assume < 32 warps
__global__ void __launch_bounds__(kEngineThreads) engine_kernel(NetDev N, EngineCtl* E, Params P);
__global__ void __launch_bounds__(kEngineThreads, 2) fc_batch_kernel(FcJob* jobs, int n_jobs,
                                                                  BatchCtl* B, int G, int Gb,
                                                                  int big, int n_groups,
                                                                  Params P0, int cluster);
// A barrier wait that only its timeout ends (which: 0 grid, 1 group in
// global memory, 2 cluster); hfp_ctx_wait_selftest launches it.
__global__ void wait_selftest_kernel(EngineCtl* E, BatchCtl* B, int which,
                                     unsigned long long timeout_ns);
// Largest group of fc_batch_kernel launched as one thread-block cluster
// (non-portable cluster size); larger groups use a cooperative launch.
constexpr int kMaxClusterCtas = 16;

// cuts.cu
enum SetupMode : int { SETUP_GR = 0, SETUP_ROUND = 1, SETUP_SR = 2, SETUP_PREP = 3, SETUP_DIST = 4,
                       SETUP_BATCH = 5, SETUP_SR_ADD = 6, SETUP_GR_ADD = 7 };
void launch_engine_setup(EngineCtl* E, int mode, cudaStream_t st, int32_t arg = 0);
void launch_saturate(const NetDev& N, EngineCtl* E, const int32_t* nodes, int32_t count,
                     cudaStream_t st);
void launch_mark_sources(const NetDev& N, EngineCtl* E, const int32_t* extra, int32_t count,
                         int sms, cudaStream_t st);
void launch_mark_sinks(const NetDev& N, EngineCtl* E, const int32_t* extra, int32_t count,
                       int sms, cudaStream_t st);
// Largest piercing key (and its node) among the candidates, or among those
// with a key below `below` when it is not 0.
void launch_pierce_select(const NetDev& N, EngineCtl* E, int grow_s, long long max_w,
                          long long w_reach, uint32_t seed, int sms, cudaStream_t st,
                          unsigned long long below = 0);
void launch_region_side(const NetDev& N, int use_t, int32_t n_region, uint8_t* out, int sms,
                        cudaStream_t st);
void launch_lawler_sink_side(const NetDev& N, uint8_t* out, int sms, cudaStream_t st);
void launch_cut_net_flags(const NetDev& N, unsigned* flags, int sms, cudaStream_t st);
void launch_cut_net_compact(const NetDev& N, const unsigned* flags, const unsigned* pos,
                            const int32_t* net_gid, int32_t* out, int32_t cap, int sms,
                            cudaStream_t st);
void launch_inc_slots(const NetDev& N, int32_t* out, int sms, cudaStream_t st);
void launch_add_i64(const long long* a, const long long* b, long long* out, long long n, int sms,
                    cudaStream_t st);

}  // namespace hfp
