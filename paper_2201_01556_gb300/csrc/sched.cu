// Learned block-pair scheduler.  The paper refines every edge of the quotient
// graph in each round (Section 5, "Quotient Graph Construction", "Parallel
// Scheduling"); this file scores the edges with a 16 -> 64 -> 64 -> 1
// perceptron so that a round can skip pairs unlikely to reduce (lambda - 1).
// It has no counterpart in the paper.
//
//   pair features   one warp per net gathers its block set (64-bit mask) and
//                   adds the net to the statistics of every block pair in it;
//                   one CTA turns the statistics into 16 floats per pair.
//   forward         bf16 tensor-core tiles (mma.sync m16n8k16, fp32
//                   accumulate): one warp per 16 rows, weights rounded to
//                   bf16 (nearest even) and staged in shared memory; the
//                   layer-1 accumulators become the layer-2 A fragments in
//                   registers.  The whole product is ~19 kFLOP per row: the
//                   kernel is bound by launch latency, not by the tensor pipe,
//                   which is why it stays on warp-level mma.
//   backward        fp32 on the CUDA cores (gradients keep fp32 accuracy):
//                   one CTA per 64 rows writes its partial gradient; a second
//                   kernel sums the partials in CTA order (deterministic) and
//                   applies Adam.  Training replays these two kernels from a
//                   CUDA graph.
#include <cmath>
#include <cstring>
#include <vector>

#include <cuda_bf16.h>

#include "internal.h"

using namespace hfp;

namespace {

constexpr int kF = HFP_MLP_FEATURES;   // 16
constexpr int kH = HFP_MLP_HIDDEN;     // 64
constexpr int kP = HFP_MLP_PARAMS;     // 5313
constexpr int OFF_W1 = 0, OFF_B1 = kH * kF, OFF_W2 = OFF_B1 + kH, OFF_B2 = OFF_W2 + kH * kH,
              OFF_W3 = OFF_B2 + kH, OFF_B3 = OFF_W3 + kH;
static_assert(OFF_B3 + 1 == kP, "parameter layout");
constexpr int kRowsPerCta = 64;        // 4 warps x 16 rows
constexpr int kMlpThreads = 128;
constexpr int kStats = 8;

inline unsigned nblk(long long work, unsigned per, unsigned cap) {
  long long b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// ---------------------------------------------------------------------------
// features

// Statistics of every block pair i < j over the nets whose blocks include
// both: 0 nets, 1 weight, 2 pins, 3 largest size, 4..6 the same three for the
// nets whose blocks are exactly {i, j}.
__global__ void k_pair_stats(int32_t m, const uint32_t* net_off, const int32_t* pins,
                             const int32_t* net_w, const int32_t* part, int32_t k,
                             unsigned long long* st) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned nw = (gridDim.x * blockDim.x) >> 5;
  for (unsigned e = gw; e < (unsigned)m; e += nw) {
    const unsigned b0 = net_off[e], b1 = net_off[e + 1];
    unsigned long long mask = 0;
    for (unsigned j = b0 + lane; j < b1; j += 32) mask |= 1ull << part[pins[j]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mask |= __shfl_xor_sync(0xffffffffu, mask, o);
    const int lam = __popcll(mask);
    if (lam < 2) continue;
    const unsigned long long size = b1 - b0, w = (unsigned long long)net_w[e];
    for (int a = lane; a < k; a += 32) {
      if (!((mask >> a) & 1ull)) continue;
      unsigned long long rest = a + 1 < 64 ? mask >> (a + 1) : 0ull;
      while (rest) {
        const int b = a + __ffsll((long long)rest);
        rest &= rest - 1;
        unsigned long long* s = st + ((size_t)a * k + b) * kStats;
        atomicAdd(s + 0, 1ull);
        atomicAdd(s + 1, w);
        atomicAdd(s + 2, size);
        atomicMax(s + 3, size);
        if (lam == 2) {
          atomicAdd(s + 4, 1ull);
          atomicAdd(s + 5, w);
          atomicAdd(s + 6, size);
        }
      }
    }
  }
}

__global__ void k_block_weight(int32_t n, const int32_t* part, const int32_t* node_w,
                               unsigned long long* bw) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    atomicAdd(&bw[part[v]], (unsigned long long)node_w[v]);
}

// One CTA of 1024 threads: thread t owns the row-major entries 4t .. 4t+3 of
// the k x k table, so a block scan numbers the pairs i < j with a joining net
// in row-major order.
__global__ void __launch_bounds__(1024) k_pair_features(
    int32_t k, const unsigned long long* st, const unsigned long long* bw, float L,
    const long long* prev, float* feat, int32_t* pairs, int32_t cap, int32_t* n_pairs) {
  __shared__ unsigned warp_cnt[32];
  __shared__ unsigned long long warp_w[32];
  __shared__ unsigned total_pairs;
  __shared__ unsigned long long total_w;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int kk = k * k;
  unsigned cnt = 0;
  unsigned long long wsum = 0;
  for (int q = 0; q < 4; q++) {
    const int idx = 4 * t + q;
    if (idx >= kk) break;
    const int i = idx / k, j = idx % k;
    if (i < j && st[(size_t)idx * kStats] > 0) {
      cnt++;
      wsum += st[(size_t)idx * kStats + 1];
    }
  }
  // inclusive warp scan of cnt, warp sums of the weight
  unsigned inc = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  unsigned long long ws = wsum;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ws += __shfl_xor_sync(0xffffffffu, ws, o);
  if (lane == 31) warp_cnt[wid] = inc;
  if (lane == 0) warp_w[wid] = ws;
  __syncthreads();
  if (wid == 0) {
    unsigned c = warp_cnt[lane];
    unsigned long long w = warp_w[lane];
    unsigned ci = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, ci, o);
      if (lane >= o) ci += y;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
    warp_cnt[lane] = ci - c;       // exclusive prefix of the warps
    if (lane == 31) total_pairs = ci;
    if (lane == 0) total_w = w;
  }
  __syncthreads();
  unsigned pos = warp_cnt[wid] + inc - cnt;
  const unsigned P = total_pairs;
  const float tot = (float)total_w, fP = (float)P;
  if (t == 0) *n_pairs = (int32_t)P;
  for (int q = 0; q < 4; q++) {
    const int idx = 4 * t + q;
    if (idx >= kk) break;
    const int i = idx / k, j = idx % k;
    if (!(i < j && st[(size_t)idx * kStats] > 0)) continue;
    const unsigned r = pos++;
    if ((int)r >= cap) continue;
    const unsigned long long* s = st + (size_t)idx * kStats;
    const long long pv = prev ? prev[idx] : -1;
    float* f = feat + (size_t)r * kF;
    f[0] = log1pf((float)s[0]);
    f[1] = log1pf((float)s[1]);
    f[2] = log1pf((float)s[2]);
    f[3] = log1pf((float)s[3]);
    f[4] = log1pf((float)s[4]);
    f[5] = log1pf((float)s[5]);
    f[6] = (float)s[5] / (float)s[1];
    f[7] = log1pf((float)s[6]);
    f[8] = (float)bw[i] / L;
    f[9] = (float)bw[j] / L;
    f[10] = (float)(bw[i] + bw[j]) / (2.0f * L);
    f[11] = log1pf((float)s[2] / (float)s[0]);
    f[12] = log1pf((float)(pv > 0 ? pv : 0));
    f[13] = pv >= 0 ? 1.0f : 0.0f;
    f[14] = log2f((float)k) / 6.0f;
    f[15] = (float)s[1] * fP / tot;
    pairs[2 * r] = i;
    pairs[2 * r + 1] = j;
  }
}

// scores of the P pairs into a k x k table (-1 where there is no pair)
__global__ void k_scatter_scores(int32_t P, const int32_t* pairs, const float* s, int32_t k,
                                 float* table) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  for (int q = t; q < k * k; q += gridDim.x * blockDim.x) table[q] = -1.0f;
  __syncthreads();
  // single CTA: the fill above and the scatter below are ordered by the barrier
  for (int r = t; r < P; r += blockDim.x) table[pairs[2 * r] * k + pairs[2 * r + 1]] = s[r];
}

// ---------------------------------------------------------------------------
// the perceptron

struct MlpSmem {
  uint32_t w1p[kH][kF / 2];      // bf16 pairs along the input index
  uint32_t w2p[kH][kH / 2];
  float w2q[kH][kH];             // bf16-rounded W2 (backward)
  float w3q[kH];
  float b1[kH], b2[kH];
  float b3;
};

struct TrainSmem {
  MlpSmem w;
  float xq[kRowsPerCta][kF];     // bf16-rounded inputs
  float h1q[kRowsPerCta][kH];    // bf16-rounded layer-1 activations
  float h2[kRowsPerCta][kH];
  float da2[kRowsPerCta][kH];
  float da1[kRowsPerCta][kH];
  float dz[kRowsPerCta];
  float loss[kRowsPerCta];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ float bf16_round(float x) {
  return __bfloat162float(__float2bfloat16_rn(x));
}

__device__ void load_weights(const float* __restrict__ prm, MlpSmem& S) {
  for (int q = threadIdx.x; q < kH * kF / 2; q += blockDim.x) {
    const int o = q / (kF / 2), c = q % (kF / 2);
    S.w1p[o][c] = pack_bf16(prm[OFF_W1 + o * kF + 2 * c], prm[OFF_W1 + o * kF + 2 * c + 1]);
  }
  for (int q = threadIdx.x; q < kH * kH / 2; q += blockDim.x) {
    const int o = q / (kH / 2), c = q % (kH / 2);
    const float a = prm[OFF_W2 + o * kH + 2 * c], b = prm[OFF_W2 + o * kH + 2 * c + 1];
    S.w2p[o][c] = pack_bf16(a, b);
    S.w2q[o][2 * c] = bf16_round(a);
    S.w2q[o][2 * c + 1] = bf16_round(b);
  }
  for (int q = threadIdx.x; q < kH; q += blockDim.x) {
    S.w3q[q] = bf16_round(prm[OFF_W3 + q]);
    S.b1[q] = prm[OFF_B1 + q];
    S.b2[q] = prm[OFF_B2 + q];
  }
  if (threadIdx.x == 0) S.b3 = prm[OFF_B3];
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Forward pass of the 16 rows r0 .. r0+15 by one warp.  Fragment layout of
// m16n8k16 (g = lane / 4, t = lane % 4): A registers hold rows g / g+8 and
// columns 2t, 2t+1 (+8); B registers hold column g and rows 2t, 2t+1 (+8);
// C holds rows g / g+8, columns 2t, 2t+1.  Two adjacent 8-column C tiles are
// exactly the A fragment of one 16-wide k slice, so layer 1's output feeds
// layer 2 without leaving registers.  Returns the logits of rows g and g+8
// (valid in all four lanes of the quad).  With a TrainSmem, the
// intermediates backward needs are stored there (rows relative to rs).
template <bool kTrain>
__device__ void warp_forward(const MlpSmem& S, const float* __restrict__ x, int rows, int r0,
                             TrainSmem* T, int rs, float& z_lo, float& z_hi) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int ra = r0 + g, rb = r0 + g + 8;
  float xa[4], xb[4];
  {
    const int cols[4] = {2 * t, 2 * t + 1, 2 * t + 8, 2 * t + 9};
#pragma unroll
    for (int q = 0; q < 4; q++) {
      xa[q] = ra < rows ? x[(size_t)ra * kF + cols[q]] : 0.0f;
      xb[q] = rb < rows ? x[(size_t)rb * kF + cols[q]] : 0.0f;
      if (kTrain) {
        T->xq[rs + g][cols[q]] = bf16_round(xa[q]);
        T->xq[rs + g + 8][cols[q]] = bf16_round(xb[q]);
      }
    }
  }
  uint32_t a[4] = {pack_bf16(xa[0], xa[1]), pack_bf16(xb[0], xb[1]), pack_bf16(xa[2], xa[3]),
                   pack_bf16(xb[2], xb[3])};
  float h[8][4];
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    h[nt][0] = h[nt][1] = h[nt][2] = h[nt][3] = 0.0f;
    mma_bf16(h[nt], a, S.w1p[8 * nt + g][t], S.w1p[8 * nt + g][t + 4]);
    const int c0 = 8 * nt + 2 * t;
    h[nt][0] = fmaxf(h[nt][0] + S.b1[c0], 0.0f);
    h[nt][1] = fmaxf(h[nt][1] + S.b1[c0 + 1], 0.0f);
    h[nt][2] = fmaxf(h[nt][2] + S.b1[c0], 0.0f);
    h[nt][3] = fmaxf(h[nt][3] + S.b1[c0 + 1], 0.0f);
    if (kTrain) {
      T->h1q[rs + g][c0] = bf16_round(h[nt][0]);
      T->h1q[rs + g][c0 + 1] = bf16_round(h[nt][1]);
      T->h1q[rs + g + 8][c0] = bf16_round(h[nt][2]);
      T->h1q[rs + g + 8][c0 + 1] = bf16_round(h[nt][3]);
    }
  }
  uint32_t a2[4][4];
#pragma unroll
  for (int s = 0; s < 4; s++) {
    a2[s][0] = pack_bf16(h[2 * s][0], h[2 * s][1]);
    a2[s][1] = pack_bf16(h[2 * s][2], h[2 * s][3]);
    a2[s][2] = pack_bf16(h[2 * s + 1][0], h[2 * s + 1][1]);
    a2[s][3] = pack_bf16(h[2 * s + 1][2], h[2 * s + 1][3]);
  }
  float za = 0.0f, zb = 0.0f;
#pragma unroll
  for (int nt = 0; nt < 8; nt++) {
    float c[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int s = 0; s < 4; s++)
      mma_bf16(c, a2[s], S.w2p[8 * nt + g][8 * s + t], S.w2p[8 * nt + g][8 * s + t + 4]);
    const int c0 = 8 * nt + 2 * t;
    const float h00 = fmaxf(c[0] + S.b2[c0], 0.0f), h01 = fmaxf(c[1] + S.b2[c0 + 1], 0.0f);
    const float h10 = fmaxf(c[2] + S.b2[c0], 0.0f), h11 = fmaxf(c[3] + S.b2[c0 + 1], 0.0f);
    za = fmaf(h00, S.w3q[c0], za);
    za = fmaf(h01, S.w3q[c0 + 1], za);
    zb = fmaf(h10, S.w3q[c0], zb);
    zb = fmaf(h11, S.w3q[c0 + 1], zb);
    if (kTrain) {
      T->h2[rs + g][c0] = h00;
      T->h2[rs + g][c0 + 1] = h01;
      T->h2[rs + g + 8][c0] = h10;
      T->h2[rs + g + 8][c0 + 1] = h11;
    }
  }
  za += __shfl_xor_sync(0xffffffffu, za, 1);
  za += __shfl_xor_sync(0xffffffffu, za, 2);
  zb += __shfl_xor_sync(0xffffffffu, zb, 1);
  zb += __shfl_xor_sync(0xffffffffu, zb, 2);
  z_lo = za + S.b3;
  z_hi = zb + S.b3;
}

__device__ __forceinline__ float sigmoid_stable(float z) {
  const float e = expf(-fabsf(z));
  return z >= 0.0f ? 1.0f / (1.0f + e) : e / (1.0f + e);
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float* __restrict__ prm,
                                                             const float* __restrict__ x,
                                                             int32_t rows, float* scores) {
  __shared__ MlpSmem S;
  load_weights(prm, S);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r0 = (blockIdx.x * 4 + warp) * 16; r0 < rows; r0 += gridDim.x * kRowsPerCta) {
    float za, zb;
    warp_forward<false>(S, x, rows, r0, nullptr, 0, za, zb);
    if ((lane & 3) == 0) {
      const int g = lane >> 2;
      if (r0 + g < rows) scores[r0 + g] = sigmoid_stable(za);
      if (r0 + g + 8 < rows) scores[r0 + g + 8] = sigmoid_stable(zb);
    }
  }
}

// Forward + backward of the 64 rows of this CTA; writes the CTA's partial
// gradient (kP floats) and loss sum to part[blockIdx.x][0 .. kP].  The mean
// over all rows is folded in through dz = (sigmoid(z) - y) / rows.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_backward(const float* __restrict__ prm,
                                                              const float* __restrict__ x,
                                                              const float* __restrict__ y,
                                                              int32_t rows, float* part,
                                                              int* step) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& T = *reinterpret_cast<TrainSmem*>(smem_raw);
  if (step && blockIdx.x == 0 && threadIdx.x == 0) (*step)++;   // read by k_mlp_reduce
  load_weights(prm, T.w);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2;
  const int base = blockIdx.x * kRowsPerCta;
  const float frows = (float)rows;
  {
    float za, zb;
    warp_forward<true>(T.w, x, rows, base + warp * 16, &T, warp * 16, za, zb);
    if ((lane & 3) == 0) {
      const float zz[2] = {za, zb};
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const int rl = warp * 16 + g + 8 * h, r = base + rl;
        float dz = 0.0f, l = 0.0f;
        if (r < rows) {
          const float z = zz[h], yy = y[r];
          dz = (sigmoid_stable(z) - yy) / frows;
          l = fmaxf(z, 0.0f) - z * yy + log1pf(expf(-fabsf(z)));
        }
        T.dz[rl] = dz;
        T.loss[rl] = l;
      }
    }
  }
  __syncthreads();
  // da2 = dz * w3 on the active units of layer 2
  for (int q = threadIdx.x; q < kRowsPerCta * kH; q += blockDim.x) {
    const int r = q / kH, o = q % kH;
    T.da2[r][o] = T.h2[r][o] > 0.0f ? T.dz[r] * T.w.w3q[o] : 0.0f;
  }
  __syncthreads();
  // da1 = (da2 W2) on the active units of layer 1
  for (int q = threadIdx.x; q < kRowsPerCta * kH; q += blockDim.x) {
    const int r = q / kH, i = q % kH;
    float acc = 0.0f;
    if (T.h1q[r][i] > 0.0f)
      for (int o = 0; o < kH; o++) acc = fmaf(T.da2[r][o], T.w.w2q[o][i], acc);
    T.da1[r][i] = acc;
  }
  __syncthreads();
  float* out = part + (size_t)blockIdx.x * (kP + 1);
  for (int q = threadIdx.x; q < kH * kH; q += blockDim.x) {
    const int o = q / kH, i = q % kH;
    float acc = 0.0f;
    for (int r = 0; r < kRowsPerCta; r++) acc = fmaf(T.da2[r][o], T.h1q[r][i], acc);
    out[OFF_W2 + q] = acc;
  }
  for (int q = threadIdx.x; q < kH * kF; q += blockDim.x) {
    const int o = q / kF, i = q % kF;
    float acc = 0.0f;
    for (int r = 0; r < kRowsPerCta; r++) acc = fmaf(T.da1[r][o], T.xq[r][i], acc);
    out[OFF_W1 + q] = acc;
  }
  for (int o = threadIdx.x; o < kH; o += blockDim.x) {
    float s1 = 0.0f, s2 = 0.0f, s3 = 0.0f;
    for (int r = 0; r < kRowsPerCta; r++) {
      s1 += T.da1[r][o];
      s2 += T.da2[r][o];
      s3 = fmaf(T.h2[r][o], T.dz[r], s3);
    }
    out[OFF_B1 + o] = s1;
    out[OFF_B2 + o] = s2;
    out[OFF_W3 + o] = s3;
  }
  if (threadIdx.x == 0) {
    float sd = 0.0f, sl = 0.0f;
    for (int r = 0; r < kRowsPerCta; r++) {
      sd += T.dz[r];
      sl += T.loss[r];
    }
    out[OFF_B3] = sd;
    out[kP] = sl;
  }
}

struct AdamArgs {
  float lr, eps, c1, c2;         // c1 = 1 - beta1, c2 = 1 - beta2 (rounded on the host)
  float beta1, beta2;
  double beta1_d, beta2_d;
};

// Sums the CTA partials in CTA order; mode 0 writes the gradient and the
// mean loss, mode 1 applies one Adam step (step number *step, 1-based) and
// records the mean loss in losses[*step - *step0 - 1] (*step0: the counter
// when the training call began).
__global__ void k_mlp_reduce(const float* part, int ncta, int32_t rows, int mode, float* grad,
                             float* loss, float* prm, float* mom, float* vel, const int* step,
                             const int* step0, AdamArgs A, float* losses, int32_t loss_cap) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p > kP) return;
  float s = 0.0f;
  for (int c = 0; c < ncta; c++) s += part[(size_t)c * (kP + 1) + p];
  if (p == kP) {
    const float mean = s / (float)rows;
    if (mode == 0) {
      if (loss) *loss = mean;
    } else if (losses && *step - *step0 - 1 < loss_cap) {
      losses[*step - *step0 - 1] = mean;
    }
    return;
  }
  if (mode == 0) {
    grad[p] = s;
    return;
  }
  const int t = *step;
  const float m = A.beta1 * mom[p] + A.c1 * s;
  const float v = A.beta2 * vel[p] + A.c2 * s * s;
  mom[p] = m;
  vel[p] = v;
  const float bc1 = (float)(1.0 - pow(A.beta1_d, (double)t));
  const float bc2 = (float)(1.0 - pow(A.beta2_d, (double)t));
  const float mh = m / bc1, vh = v / bc2;
  prm[p] = prm[p] - A.lr * mh / (sqrtf(vh) + A.eps);
}

hfp_status set_dev(hfp_ctx* ctx) {
  CK(cudaSetDevice(ctx->device));
  return HFP_OK;
}

hfp_status ensure_train_smem() {
  static bool done = false;
  if (!done) {
    CK(cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)sizeof(TrainSmem)));
    done = true;
  }
  return HFP_OK;
}

// forward + backward partials of all rows (one launch)
hfp_status launch_backward(hfp_ctx* ctx, const float* prm, const float* x, const float* y,
                           int32_t rows, float* part, int* step, cudaStream_t st) {
  const int ncta = (rows + kRowsPerCta - 1) / kRowsPerCta;
  k_mlp_backward<<<ncta, kMlpThreads, sizeof(TrainSmem), st>>>(prm, x, y, rows, part, step);
  count_launches(1);
  CK(cudaGetLastError());
  return HFP_OK;
}

hfp_status features(hfp_hgraph* hg, const int32_t* part, int32_t k, int32_t eps_pct,
                    const int64_t* prev_gain, float* feat, int32_t* pairs, int32_t cap,
                    int32_t* n_pairs) {
  hfp_ctx* ctx = hg->ctx;
  cudaStream_t st = ctx->stream;
  const int sms = ctx->sms;
  DevBuf stats, bw, prev, np;
  CK(stats.alloc(sizeof(unsigned long long) * k * k * kStats, st));
  CK(bw.alloc(sizeof(unsigned long long) * k, st));
  CK(np.alloc(sizeof(int32_t), st));
  CK(cudaMemsetAsync(stats.p, 0, sizeof(unsigned long long) * k * k * kStats, st));
  CK(cudaMemsetAsync(bw.p, 0, sizeof(unsigned long long) * k, st));
  if (prev_gain) {
    CK(prev.alloc(sizeof(long long) * k * k, st));
    CK(cudaMemcpyAsync(prev.p, prev_gain, sizeof(long long) * k * k, cudaMemcpyHostToDevice, st));
  }
  if (hg->m) {
    k_pair_stats<<<nblk((long long)hg->m * 32, 256, sms * 16), 256, 0, st>>>(
        hg->m, hg->net_off, hg->pins, hg->net_w, part, k, stats.as<unsigned long long>());
    count_launches(1);
  }
  if (hg->n) {
    k_block_weight<<<nblk(hg->n, 256, sms * 8), 256, 0, st>>>(hg->n, part, hg->node_w,
                                                              bw.as<unsigned long long>());
    count_launches(1);
  }
  const long long L = ((100 + eps_pct) * ((hg->total_w + k - 1) / k)) / 100;
  k_pair_features<<<1, 1024, 0, st>>>(k, stats.as<unsigned long long>(),
                                      bw.as<unsigned long long>(), (float)L, prev.as<long long>(),
                                      feat, pairs, cap, np.as<int32_t>());
  count_launches(1);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(n_pairs, np.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}

}  // namespace

HFP_API hfp_status hfp_pair_features(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                     int32_t eps_pct, const int64_t* prev_gain, float* features_,
                                     int32_t* pairs, int32_t cap, int32_t* n_pairs) {
  if (!hg || !part || !n_pairs || k < 2 || k > 64 || eps_pct < 0 || cap < 0 ||
      (cap > 0 && (!features_ || !pairs)))
    return fail(HFP_ERR_INVALID, "bad arguments");
  hfp_status s = set_dev(hg->ctx);
  if (s != HFP_OK) return s;
  if ((s = features(hg, part, k, eps_pct, prev_gain, features_, pairs, cap, n_pairs)) != HFP_OK)
    return s;
  if (*n_pairs > cap) return fail(HFP_ERR_BUFFER_TOO_SMALL, "%d pairs", *n_pairs);
  return HFP_OK;
}

HFP_API hfp_status hfp_mlp_forward(hfp_ctx* ctx, const float* params, const float* x,
                                   int32_t rows, float* scores) {
  if (!ctx || rows < 0 || (rows > 0 && (!params || !x || !scores)))
    return fail(HFP_ERR_INVALID, "bad arguments");
  if (rows == 0) return HFP_OK;
  hfp_status s = set_dev(ctx);
  if (s != HFP_OK) return s;
  const unsigned ncta = (unsigned)((rows + kRowsPerCta - 1) / kRowsPerCta);
  k_mlp_forward<<<ncta, kMlpThreads, 0, ctx->stream>>>(params, x, rows, scores);
  count_launches(1);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(ctx->stream));
  return HFP_OK;
}

HFP_API hfp_status hfp_mlp_grad(hfp_ctx* ctx, const float* params, const float* x,
                                const float* y, int32_t rows, float* grad, float* loss) {
  if (!ctx || rows <= 0 || !params || !x || !y || !grad)
    return fail(HFP_ERR_INVALID, "bad arguments");
  hfp_status s = set_dev(ctx);
  if (s != HFP_OK) return s;
  if ((s = ensure_train_smem()) != HFP_OK) return s;
  cudaStream_t st = ctx->stream;
  const int ncta = (rows + kRowsPerCta - 1) / kRowsPerCta;
  DevBuf part, l;
  CK(part.alloc(sizeof(float) * (size_t)ncta * (kP + 1), st));
  CK(l.alloc(sizeof(float), st));
  if ((s = launch_backward(ctx, params, x, y, rows, part.as<float>(), nullptr, st)) != HFP_OK)
    return s;
  k_mlp_reduce<<<(kP + 1 + 255) / 256, 256, 0, st>>>(part.as<float>(), ncta, rows, 0, grad,
                                                     l.as<float>(), nullptr, nullptr, nullptr,
                                                     nullptr, nullptr, AdamArgs{}, nullptr, 0);
  count_launches(1);
  CK(cudaGetLastError());
  float h = 0.0f;
  CK(cudaMemcpyAsync(&h, l.p, sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (loss) *loss = h;
  return HFP_OK;
}

HFP_API hfp_status hfp_mlp_train(hfp_ctx* ctx, float* params, float* adam_m, float* adam_v,
                                 int32_t* step, const float* x, const float* y, int32_t rows,
                                 int32_t steps, const hfp_adam_params* opt, float* losses,
                                 int32_t loss_cap) {
  if (!ctx || !params || !adam_m || !adam_v || !step || !x || !y || !opt || rows <= 0 ||
      steps < 0 || loss_cap < 0 || (loss_cap > 0 && !losses))
    return fail(HFP_ERR_INVALID, "bad arguments");
  if (!(opt->beta1 >= 0 && opt->beta1 < 1 && opt->beta2 >= 0 && opt->beta2 < 1 && opt->lr > 0 &&
        opt->eps > 0))
    return fail(HFP_ERR_INVALID, "bad Adam parameters");
  if (steps == 0) return HFP_OK;
  hfp_status s = set_dev(ctx);
  if (s != HFP_OK) return s;
  if ((s = ensure_train_smem()) != HFP_OK) return s;
  cudaStream_t st = ctx->stream;
  const int ncta = (rows + kRowsPerCta - 1) / kRowsPerCta;
  DevBuf part, step0;
  CK(part.alloc(sizeof(float) * (size_t)ncta * (kP + 1), st));
  CK(step0.alloc(sizeof(int), st));
  CK(cudaMemcpyAsync(step0.p, step, sizeof(int), cudaMemcpyDeviceToDevice, st));
  AdamArgs A;
  A.lr = opt->lr;
  A.eps = opt->eps;
  A.beta1 = (float)opt->beta1;
  A.beta2 = (float)opt->beta2;
  A.c1 = (float)(1.0 - opt->beta1);
  A.c2 = (float)(1.0 - opt->beta2);
  A.beta1_d = opt->beta1;
  A.beta2_d = opt->beta2;
  // one step = backward partials + reduce/Adam, captured once and replayed
  cudaStream_t cs = nullptr;
  cudaEvent_t ev = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  auto cleanup = [&]() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev) cudaEventDestroy(ev);
    if (cs) cudaStreamDestroy(cs);
  };
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(ev, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev, 0);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    k_mlp_backward<<<ncta, kMlpThreads, sizeof(TrainSmem), cs>>>(params, x, y, rows,
                                                                 part.as<float>(), step);
    k_mlp_reduce<<<(kP + 1 + 255) / 256, 256, 0, cs>>>(part.as<float>(), ncta, rows, 1, nullptr,
                                                       nullptr, params, adam_m, adam_v, step,
                                                       step0.as<int>(), A, losses, loss_cap);
    cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
    e = e2 != cudaSuccess ? e2 : cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  for (int32_t i = 0; e == cudaSuccess && i < steps; i++) {
    e = cudaGraphLaunch(exec, cs);
    count_launches(2);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ev, 0);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess)
    return fail(e == cudaErrorMemoryAllocation ? HFP_ERR_OOM : HFP_ERR_CUDA, "training: %s",
                cudaGetErrorString(e));
  return HFP_OK;
}

HFP_API hfp_status hfp_pair_scores(hfp_hgraph* hg, const int32_t* part, int32_t k,
                                   int32_t eps_pct, const int64_t* prev_gain, const float* params,
                                   float* scores) {
  if (!hg || !part || !params || !scores || k < 2 || k > 64 || eps_pct < 0)
    return fail(HFP_ERR_INVALID, "bad arguments");
  hfp_status s = set_dev(hg->ctx);
  if (s != HFP_OK) return s;
  cudaStream_t st = hg->ctx->stream;
  const int cap = k * (k - 1) / 2;
  DevBuf feat, pairs, sc, table;
  CK(feat.alloc(sizeof(float) * cap * kF, st));
  CK(pairs.alloc(sizeof(int32_t) * cap * 2, st));
  CK(sc.alloc(sizeof(float) * cap, st));
  CK(table.alloc(sizeof(float) * k * k, st));
  int32_t P = 0;
  if ((s = features(hg, part, k, eps_pct, prev_gain, feat.as<float>(), pairs.as<int32_t>(), cap,
                    &P)) != HFP_OK)
    return s;
  if (P > 0) {
    k_mlp_forward<<<(P + kRowsPerCta - 1) / kRowsPerCta, kMlpThreads, 0, st>>>(
        params, feat.as<float>(), P, sc.as<float>());
    count_launches(1);
  }
  k_scatter_scores<<<1, 1024, 0, st>>>(P, pairs.as<int32_t>(), sc.as<float>(), k,
                                       table.as<float>());
  count_launches(1);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(scores, table.p, sizeof(float) * k * k, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return HFP_OK;
}
