// gn_mpnn.cu -- the learned warm start: a message-passing network that predicts x0 for GN,
// trained on converged GN states by these forward and backward kernels.
//
// Network (per vertex i, N(i) its neighbours):
//   features  f_i = [log w_i, log(1 + deg_i), mean_{N(i)} log w_j, max_{N(i)} log w_j]
//   layer l   z^l_i = W_s^l h^{l-1}_i + W_n^l mean_{j in N(i)} h^{l-1}_j + b^l,  h^l = relu(z^l)
//   head      q_i = w_o . h^L_i + b_o,  p_i = sigmoid(q_i),  x0_i = clamp(p_i, 1e-3, 1)
//   loss      mean_i BCE(p_i, t_i) against the rounded converged GN state t
// Weights live as FP32 masters and are rounded to bf16 for every forward and backward pass;
// activations and accumulation are FP32.  The dense part is a 128 x 64 product per vertex, so
// the layer is bound by reading activations, not by arithmetic: it runs on the FP32 pipes with
// the bf16 weights staged in shared memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gn_internal.cuh"

namespace gn {

static constexpr int kF = 4;      // input features
static constexpr int kH = 64;     // hidden width
static constexpr int kL = 3;      // layers
static constexpr int kRows = 32;  // rows per tile in the dense kernels
static constexpr int kHeadRows = 128;  // rows (threads) per CTA of the head
static constexpr int kDenseThreads = 128;            // threads of the forward dense kernel
static constexpr int kDenseRows = 8 * kDenseThreads / 8;  // its rows per tile: 8 per thread, 8 threads per row group

__host__ __device__ constexpr int layer_in(int l) { return l == 0 ? kF : kH; }
// parameter layout (FP32): per layer Ws [kH x din], Wn [kH x din], b [kH]; then wo [kH], bo [1]
__host__ __device__ constexpr int layer_off(int l) {
  return l == 0 ? 0 : layer_off(l - 1) + 2 * kH * layer_in(l - 1) + kH;
}
static constexpr int kNumParams = layer_off(kL) + kH + 1;

__global__ void k_features(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const float* __restrict__ w, float* __restrict__ X) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int a = rp[i], b = rp[i + 1];
  float mean = 0.0f, mx = 0.0f;
  for (int e = a; e < b; ++e) {
    const float lw = logf(w[ci[e]]);
    mean += lw;
    mx = e == a ? lw : fmaxf(mx, lw);
  }
  if (b > a) mean /= (float)(b - a);
  X[(size_t)i * kF + 0] = logf(w[i]);
  X[(size_t)i * kF + 1] = logf(1.0f + (float)(b - a));
  X[(size_t)i * kF + 2] = mean;
  X[(size_t)i * kF + 3] = mx;
}

// M_i = mean_{j in N(i)} H_j (0 for an isolated vertex), each feature summed over the
// neighbours in CSR order.  D = kF (4 features): a thread per vertex, one 16-byte load per
// neighbour.  D = kH: a warp per vertex, lane l owning features l and l + 32; the lanes read 32
// neighbour ids at once and broadcast them, and four neighbours' rows are loaded before they
// are added (in order).
template <int D>
__global__ void k_aggregate(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                            const float* __restrict__ H, float* __restrict__ M) {
  static_assert(D == kF || D == kH, "aggregation widths");
  if (D == kF) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int a = rp[i], b = rp[i + 1];
    const float inv = b > a ? 1.0f / (float)(b - a) : 0.0f;
    float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    for (int e = a; e < b; ++e) {
      const float4 h = reinterpret_cast<const float4*>(H)[ci[e]];
      s.x += h.x;
      s.y += h.y;
      s.z += h.z;
      s.w += h.w;
    }
    reinterpret_cast<float4*>(M)[i] = make_float4(s.x * inv, s.y * inv, s.z * inv, s.w * inv);
    return;
  }
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  const int a = rp[i], b = rp[i + 1];
  const float inv = b > a ? 1.0f / (float)(b - a) : 0.0f;
  float s0 = 0.0f, s1 = 0.0f;
  for (int base = a; base < b; base += 32) {
    const int cnt = min(32, b - base);
    const int mine = lane < cnt ? ci[base + lane] : 0;
    int t = 0;
    for (; t + 4 <= cnt; t += 4) {
      float h0[4], h1[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = __shfl_sync(0xffffffffu, mine, t + u);
        h0[u] = H[(size_t)j * D + lane];
        h1[u] = H[(size_t)j * D + lane + 32];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        s0 += h0[u];
        s1 += h1[u];
      }
    }
    for (; t < cnt; ++t) {
      const int j = __shfl_sync(0xffffffffu, mine, t);
      s0 += H[(size_t)j * D + lane];
      s1 += H[(size_t)j * D + lane + 32];
    }
  }
  M[(size_t)i * D + lane] = s0 * inv;
  M[(size_t)i * D + lane + 32] = s1 * inv;
}

// the transpose: dH_j += sum_{i in N(j)} dM_i / deg_i (A symmetric)
template <int D>
__global__ void k_aggregate_t(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                              const float* __restrict__ dM, float* __restrict__ dH) {
  const int j = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (j >= n) return;
  const int a = rp[j], b = rp[j + 1];
  for (int f = lane; f < D; f += 32) {
    float s = 0.0f;
    for (int e = a; e < b; ++e) {
      const int i = ci[e];
      s += dM[(size_t)i * D + f] / (float)(rp[i + 1] - rp[i]);
    }
    dH[(size_t)j * D + f] += s;
  }
}

// Z = H Ws^T + M Wn^T + b, Hout = relu(Z).  The CTA stages the layer's weights once and walks
// tiles of kDenseRows rows (grid-stride) staged in shared memory (dynamic, [rows][2 DIN + 1]).
// 128 threads; thread (c, g) computes rows 8g..8g+7 of the tile at outputs c, c + 8, ..., c + 56,
// so each weight and each input read from shared memory feeds eight FMAs (the bank of a read
// is c + 8q + k or 8g + i + k mod 32: no conflicts), and consecutive threads store consecutive
// outputs.  Every output is the same FMA chain over k as a plain dot product.  Z is kept only
// for training (nullptr: inference).
template <int DIN>
__global__ void __launch_bounds__(kDenseThreads) k_dense_fwd(int n, const float* __restrict__ H,
                                                             const float* __restrict__ M,
                                                             const __nv_bfloat16* __restrict__ Wb,
                                                             float* __restrict__ Z, float* __restrict__ Hout) {
  __shared__ float sW[2][kH][DIN + 1];
  __shared__ float sb[kH];
  extern __shared__ float sXd[];
  float(*sX)[2 * DIN + 1] = reinterpret_cast<float(*)[2 * DIN + 1]>(sXd);
  for (int t = threadIdx.x; t < 2 * kH * DIN; t += blockDim.x) {
    const int m = t / (kH * DIN), rem = t % (kH * DIN);
    sW[m][rem / DIN][rem % DIN] = __bfloat162float(Wb[t]);
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) sb[t] = __bfloat162float(Wb[2 * kH * DIN + t]);
  const int c = threadIdx.x & 7, g = threadIdx.x >> 3;
  const int ntiles = (n + kDenseRows - 1) / kDenseRows;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int r0 = tile * kDenseRows;
    __syncthreads();  // the weights (first tile) / the previous tile's reads of sX
    for (int t = threadIdx.x; t < kDenseRows * DIN; t += blockDim.x) {
      const int r = t / DIN, k = t % DIN;
      const bool in = r0 + r < n;
      sX[r][k] = in ? H[(size_t)(r0 + r) * DIN + k] : 0.0f;
      sX[r][DIN + k] = in ? M[(size_t)(r0 + r) * DIN + k] : 0.0f;
    }
    __syncthreads();
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[i][q] = sb[c + 8 * q];
    for (int k = 0; k < DIN; ++k) {
      float h[8], mm[8], ws[8], wn[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        h[i] = sX[8 * g + i][k];
        mm[i] = sX[8 * g + i][DIN + k];
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        ws[q] = sW[0][c + 8 * q][k];
        wn[q] = sW[1][c + 8 * q][k];
      }
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[i][q] = fmaf(ws[q], h[i], fmaf(wn[q], mm[i], acc[i][q]));
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int r = r0 + 8 * g + i;
      if (r < n) {
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          if (Z) Z[(size_t)r * kH + c + 8 * q] = acc[i][q];
          Hout[(size_t)r * kH + c + 8 * q] = fmaxf(acc[i][q], 0.0f);
        }
      }
    }
  }
}
template <int DIN>
constexpr size_t dense_fwd_smem() { return sizeof(float) * (size_t)kDenseRows * (2 * DIN + 1); }

// ---- the hidden layers (DIN = kH) on the tensor cores: Z = [H | M] W^T + b as a GEMM with
// K = 2 kH = 128 and N = kH = 64, mma.sync m16n8k16 with bf16 operands and FP32 accumulation.
// The weights are bf16 already (exact operands).  Each FP32 activation a is split into
// a_hi = bf16(a) and a_lo = bf16(a - a_hi), and both halves are multiplied: the operand keeps
// about 16 bits (|a - a_hi - a_lo| <= 2^-17 |a|), so the layer stays at FP32-grade precision
// instead of rounding the activations to bf16.  A warp computes 16 rows x 64 outputs (eight n8
// tiles, 32 accumulators per thread) from fragments loaded straight from global memory (each
// 16-byte-per-row request fills whole 32-byte sectors); the weights sit in shared memory,
// rows padded so that a fragment's 32 words fall in 32 banks.
static constexpr int kTcWarps = 4;                 // warps per CTA, 16 rows each
static constexpr int kTcRows = 16 * kTcWarps;      // rows per CTA tile
static constexpr int kTcK = 2 * kH;                // [H | M]
static constexpr int kTcPad = kTcK + 8;            // bf16 per weight row in shared memory

__device__ __forceinline__ uint32_t pack_bf16x2(float lo_elem, float hi_elem) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);  // .x (low half) = lo_elem
  return *reinterpret_cast<const uint32_t*>(&v);
}
// split two FP32 values into their bf16 high parts and the bf16 rounding of the remainders
__device__ __forceinline__ void split_bf16x2(float2 a, uint32_t& hi, uint32_t& lo) {
  const float hx = __bfloat162float(__float2bfloat16_rn(a.x));
  const float hy = __bfloat162float(__float2bfloat16_rn(a.y));
  hi = pack_bf16x2(hx, hy);
  lo = pack_bf16x2(a.x - hx, a.y - hy);
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ float2 load_pair(const float* __restrict__ X, int row, int col, int n) {
  return row < n ? *reinterpret_cast<const float2*>(X + (size_t)row * kH + col) : make_float2(0.0f, 0.0f);
}

__global__ void __launch_bounds__(32 * kTcWarps) k_dense_fwd_tc(int n, const float* __restrict__ H,
                                                                const float* __restrict__ M,
                                                                const __nv_bfloat16* __restrict__ Wb,
                                                                float* __restrict__ Z, float* __restrict__ Hout) {
  __shared__ __align__(16) __nv_bfloat16 sW[kH][kTcPad];  // W[o][k], k over [Ws | Wn]
  __shared__ float sb[kH];
  for (int t = threadIdx.x; t < 2 * kH * kH; t += blockDim.x) {
    const int m = t / (kH * kH), rem = t % (kH * kH), o = rem / kH, k = rem % kH;
    sW[o][m * kH + k] = Wb[t];
  }
  for (int t = threadIdx.x; t < kH; t += blockDim.x) sb[t] = __bfloat162float(Wb[2 * kH * kH + t]);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
  const int ntiles = (n + kTcRows - 1) / kTcRows;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int ra = tile * kTcRows + warp * 16 + g, rb = ra + 8;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      acc[j][0] = acc[j][2] = sb[8 * j + 2 * q];
      acc[j][1] = acc[j][3] = sb[8 * j + 2 * q + 1];
    }
#pragma unroll 2
    for (int ks = 0; ks < kTcK / 16; ++ks) {
      const float* __restrict__ X = ks < kH / 16 ? H : M;
      const int c = (ks & (kH / 16 - 1)) * 16 + 2 * q;
      uint32_t ahi[4], alo[4];
      split_bf16x2(load_pair(X, ra, c, n), ahi[0], alo[0]);
      split_bf16x2(load_pair(X, rb, c, n), ahi[1], alo[1]);
      split_bf16x2(load_pair(X, ra, c + 8, n), ahi[2], alo[2]);
      split_bf16x2(load_pair(X, rb, c + 8, n), ahi[3], alo[3]);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(&sW[8 * j + g][16 * ks + 2 * q]);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(&sW[8 * j + g][16 * ks + 2 * q + 8]);
        mma_bf16(acc[j], alo, b0, b1);
        mma_bf16(acc[j], ahi, b0, b1);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int col = 8 * j + 2 * q;
      if (ra < n) {
        if (Z) *reinterpret_cast<float2*>(Z + (size_t)ra * kH + col) = make_float2(acc[j][0], acc[j][1]);
        *reinterpret_cast<float2*>(Hout + (size_t)ra * kH + col) =
            make_float2(fmaxf(acc[j][0], 0.0f), fmaxf(acc[j][1], 0.0f));
      }
      if (rb < n) {
        if (Z) *reinterpret_cast<float2*>(Z + (size_t)rb * kH + col) = make_float2(acc[j][2], acc[j][3]);
        *reinterpret_cast<float2*>(Hout + (size_t)rb * kH + col) =
            make_float2(fmaxf(acc[j][2], 0.0f), fmaxf(acc[j][3], 0.0f));
      }
    }
  }
}

// dZ = dHout (.) [Z > 0]; dH = dZ Ws, dM = dZ Wn (per row); kRows rows per CTA
template <int DIN>
// (dM may alias dHout: each CTA reads its rows of dHout before the barrier and writes them after)
__global__ void __launch_bounds__(256) k_dense_bwd_data(int n, const float* dHout, const float* __restrict__ Z,
                                                        const __nv_bfloat16* __restrict__ Wb,
                                                        float* __restrict__ dZ, float* dH, float* dM) {
  __shared__ float sW[2][kH][DIN + 1];
  __shared__ float sG[kRows][kH + 1];
  const int r0 = blockIdx.x * kRows;
  for (int t = threadIdx.x; t < 2 * kH * DIN; t += blockDim.x) {
    const int m = t / (kH * DIN), rem = t % (kH * DIN);
    sW[m][rem / DIN][rem % DIN] = __bfloat162float(Wb[t]);
  }
  for (int t = threadIdx.x; t < kRows * kH; t += blockDim.x) {
    const int r = t / kH, o = t % kH;
    float gz = 0.0f;
    if (r0 + r < n) {
      const size_t idx = (size_t)(r0 + r) * kH + o;
      gz = Z[idx] > 0.0f ? dHout[idx] : 0.0f;
      dZ[idx] = gz;
    }
    sG[r][o] = gz;
  }
  __syncthreads();
  // 2 * DIN outputs per row, 8 threads per row
  const int row = threadIdx.x >> 3, sub = threadIdx.x & 7;
  if (r0 + row >= n) return;
  for (int c = sub; c < 2 * DIN; c += 8) {
    const int m = c / DIN, k = c % DIN;
    float acc = 0.0f;
    for (int o = 0; o < kH; ++o) acc = fmaf(sG[row][o], sW[m][o][k], acc);
    (m == 0 ? dH : dM)[(size_t)(r0 + row) * DIN + k] = acc;
  }
}

// weight gradients over this CTA's rows: dWs = dZ^T H, dWn = dZ^T M, db = sum dZ, into the CTA's
// own slot of part (k_reduce_parts adds the slots in CTA order, so the sum does not depend on
// the CTAs' timing)
template <int DIN>
__global__ void __launch_bounds__(256) k_dense_bwd_weight(int n, int rows_per_cta, const float* __restrict__ dZ,
                                                          const float* __restrict__ H, const float* __restrict__ M,
                                                          float* __restrict__ part) {
  __shared__ float sG[kRows][kH + 1];
  __shared__ float sX[kRows][2 * DIN + 1];
  const int rbeg = blockIdx.x * rows_per_cta, rend = min(n, rbeg + rows_per_cta);
  constexpr int NW = 2 * kH * DIN + kH;
  float acc[(NW + 255) / 256];
#pragma unroll
  for (int q = 0; q < (NW + 255) / 256; ++q) acc[q] = 0.0f;
  for (int r0 = rbeg; r0 < rend; r0 += kRows) {
    __syncthreads();
    for (int t = threadIdx.x; t < kRows * kH; t += blockDim.x) {
      const int r = t / kH, o = t % kH;
      sG[r][o] = r0 + r < rend ? dZ[(size_t)(r0 + r) * kH + o] : 0.0f;
    }
    for (int t = threadIdx.x; t < kRows * DIN; t += blockDim.x) {
      const int r = t / DIN, k = t % DIN;
      const bool in = r0 + r < rend;
      sX[r][k] = in ? H[(size_t)(r0 + r) * DIN + k] : 0.0f;
      sX[r][DIN + k] = in ? M[(size_t)(r0 + r) * DIN + k] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < (NW + 255) / 256; ++q) {
      const int p = threadIdx.x + q * 256;
      if (p >= NW) continue;
      float a = acc[q];
      if (p < 2 * kH * DIN) {
        const int m = p / (kH * DIN), rem = p % (kH * DIN), o = rem / DIN, k = rem % DIN;
        for (int r = 0; r < kRows; ++r) a = fmaf(sG[r][o], sX[r][m * DIN + k], a);
      } else {
        const int o = p - 2 * kH * DIN;
        for (int r = 0; r < kRows; ++r) a += sG[r][o];
      }
      acc[q] = a;
    }
  }
#pragma unroll
  for (int q = 0; q < (NW + 255) / 256; ++q) {
    const int p = threadIdx.x + q * 256;
    if (p < NW) part[(size_t)blockIdx.x * NW + p] = acc[q];
  }
}

// out[p] += sum over slots b < nslot of part[b * width + p], in slot order
__global__ void k_reduce_parts(int nslot, int width, const float* __restrict__ part, float* __restrict__ out) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= width) return;
  float s = 0.0f;
  for (int b = 0; b < nslot; ++b) s += part[(size_t)b * width + p];
  out[p] += s;
}

// head: q = wo . h + bo, p = sigmoid(q); BCE loss (stable form) and dq = (p - t) / n; x0 out.
// With alpha < 1 the start blends the prediction with the cold start geometrically:
// x0 = clamp((1/(deg+1))^(1-alpha) p^alpha, 1e-3, 1).
// (kHeadRows threads; the CTA's rows of H are staged in shared memory with coalesced loads)
__global__ void __launch_bounds__(kHeadRows) k_head(int n, const float* __restrict__ H,
                                                    const __nv_bfloat16* __restrict__ wo_b,
                                                    const float* __restrict__ target,
                                                    const int32_t* __restrict__ perm_int_to_caller,
                                                    float* __restrict__ x0_caller, float* __restrict__ dq,
                                                    double* __restrict__ loss, const int32_t* __restrict__ rp,
                                                    float alpha) {
  __shared__ float swo[kH + 1];
  __shared__ double sl[kHeadRows / 32];
  __shared__ float sH[kHeadRows][kH + 1];
  for (int t = threadIdx.x; t <= kH; t += blockDim.x) swo[t] = __bfloat162float(wo_b[t]);
  const int i0 = blockIdx.x * kHeadRows;
  for (int t = threadIdx.x; t < kHeadRows * kH; t += blockDim.x) {
    const int r = t / kH, k = t % kH;
    sH[r][k] = i0 + r < n ? H[(size_t)(i0 + r) * kH + k] : 0.0f;
  }
  __syncthreads();
  const int i = i0 + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    float q = swo[kH];
    for (int k = 0; k < kH; ++k) q = fmaf(swo[k], sH[threadIdx.x][k], q);
    const float p = 1.0f / (1.0f + expf(-q));
    const int c = perm_int_to_caller ? perm_int_to_caller[i] : i;
    if (x0_caller) {
      float x = p;
      if (alpha < 1.0f) {
        const float lc = -logf((float)(rp[i + 1] - rp[i] + 1));  // log of the cold start 1/(deg+1)
        x = expf((1.0f - alpha) * lc + alpha * logf(fmaxf(p, 1e-30f)));
      }
      x0_caller[c] = fminf(fmaxf(x, 1e-3f), 1.0f);
    }
    if (target) {
      const float t = target[c];
      // BCE with logits: max(q, 0) - q t + log(1 + exp(-|q|))
      l = (double)(fmaxf(q, 0.0f) - q * t + log1pf(expf(-fabsf(q))));
      dq[i] = (p - t) / (float)n;
    }
  }
  // block sum of the loss (FP64, one atomic per CTA), training only (`target` is uniform)
  if (target) {
    l = dev::warp_sum_d(l);
    if ((threadIdx.x & 31) == 0) sl[threadIdx.x >> 5] = l;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) s += sl[j];
      atomicAdd(loss, s / (double)n);
    }
  }
}

// head backward: dH3 = dq wo; this CTA's rows' dwo = sum dq h and dbo = sum dq, summed in row
// order into the CTA's slot of part (k_reduce_parts adds the slots in CTA order)
__global__ void k_head_bwd(int n, const float* __restrict__ H, const __nv_bfloat16* __restrict__ wo_b,
                           const float* __restrict__ dq, float* __restrict__ dH, float* __restrict__ part) {
  __shared__ float swo[kH];
  for (int t = threadIdx.x; t < kH; t += blockDim.x) swo[t] = __bfloat162float(wo_b[t]);
  __syncthreads();
  const int i0 = blockIdx.x * blockDim.x, i = i0 + threadIdx.x;
  if (i < n) {
    const float g = dq[i];
    for (int k = 0; k < kH; ++k) dH[(size_t)i * kH + k] = g * swo[k];
  }
  if (threadIdx.x <= kH) {
    const int k = threadIdx.x, i1 = min(n, i0 + (int)blockDim.x);
    float a = 0.0f;
    for (int r = i0; r < i1; ++r) a = fmaf(dq[r], k < kH ? H[(size_t)r * kH + k] : 1.0f, a);
    part[(size_t)blockIdx.x * (kH + 1) + k] = a;
  }
}

// Adam on the FP32 masters; the bf16 copy used by the kernels is refreshed
__global__ void k_adam(int np, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ wb, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(int np, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < np) wb[i] = __float2bfloat16_rn(w[i]);
}

__global__ void k_gather_caller(int n, const float* __restrict__ src_caller, const int32_t* __restrict__ perm,
                                float* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src_caller[perm ? perm[i] : i];
}

}  // namespace gn

struct gn_mpnn {
  int device = 0;
  int num_sms = 1;
  cudaStream_t stream = nullptr;
  float* d_w = nullptr;             // FP32 masters
  __nv_bfloat16* d_wb = nullptr;    // bf16 copy used by the kernels
  float* d_g = nullptr;             // gradients
  float* d_m = nullptr;             // Adam moments
  float* d_v = nullptr;
  int adam_t = 0;
  // activations of the last forward (for the backward), sized for cap vertices
  int cap = 0;
  int n = 0;
  float* X = nullptr;               // [n x kF]
  float* Ms[gn::kL] = {};           // aggregated inputs per layer
  float* Zs[gn::kL] = {};           // pre-activations
  float* Hs[gn::kL] = {};           // outputs
  float* dq = nullptr;
  float* tgt = nullptr;
  float* bufA = nullptr;            // [n x kH] scratch for gradients
  float* bufB = nullptr;
  float* bufC = nullptr;
  float* part = nullptr;            // per-CTA partial gradients, reduced in CTA order
  double* d_loss = nullptr;
  double* h_loss = nullptr;         // pinned
  const gn_graph* last_graph = nullptr;
};

namespace gn {

static unsigned blk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

static gn_status mpnn_reserve(gn_mpnn* m, int n) {
  if (n <= m->cap) return GN_OK;
  float** bufs[] = {&m->X, &m->dq, &m->tgt, &m->bufA, &m->bufB, &m->bufC, &m->part};
  for (float** b : bufs)
    if (*b) cudaFree(*b), *b = nullptr;
  for (int l = 0; l < kL; ++l) {
    if (m->Ms[l]) cudaFree(m->Ms[l]);
    if (m->Zs[l]) cudaFree(m->Zs[l]);
    if (m->Hs[l]) cudaFree(m->Hs[l]);
    m->Ms[l] = m->Zs[l] = m->Hs[l] = nullptr;
  }
  const size_t nh = sizeof(float) * (size_t)n * kH;
  GN_CUDA(cudaMalloc(&m->X, sizeof(float) * (size_t)n * kF));
  GN_CUDA(cudaMalloc(&m->dq, sizeof(float) * n));
  GN_CUDA(cudaMalloc(&m->tgt, sizeof(float) * n));
  GN_CUDA(cudaMalloc(&m->bufA, nh));
  GN_CUDA(cudaMalloc(&m->bufB, nh));
  GN_CUDA(cudaMalloc(&m->bufC, nh));
  {  // the weight gradients' partials: a slot of the widest layer's size per 256 rows
    constexpr int kNWmax = 2 * kH * (kF > kH ? kF : kH) + kH;
    GN_CUDA(cudaMalloc(&m->part, sizeof(float) * (size_t)blk(n, 256) * kNWmax));
  }
  for (int l = 0; l < kL; ++l) {
    GN_CUDA(cudaMalloc(&m->Ms[l], sizeof(float) * (size_t)n * layer_in(l)));
    GN_CUDA(cudaMalloc(&m->Zs[l], nh));
    GN_CUDA(cudaMalloc(&m->Hs[l], nh));
  }
  m->cap = n;
  return GN_OK;
}


}  // namespace gn

extern "C" int gn_mpnn_num_params(void) { return gn::kNumParams; }

extern "C" void gn_mpnn_destroy(gn_mpnn* m) {
  if (!m) return;
  cudaSetDevice(m->device);
  if (m->stream) cudaStreamSynchronize(m->stream);
  void* d[] = {m->d_w, m->d_wb, m->d_g, m->d_m, m->d_v, m->X, m->dq, m->tgt, m->bufA, m->bufB, m->bufC, m->part,
               m->d_loss};
  for (void* p : d)
    if (p) cudaFree(p);
  for (int l = 0; l < gn::kL; ++l) {
    if (m->Ms[l]) cudaFree(m->Ms[l]);
    if (m->Zs[l]) cudaFree(m->Zs[l]);
    if (m->Hs[l]) cudaFree(m->Hs[l]);
  }
  if (m->h_loss) cudaFreeHost(m->h_loss);
  delete m;
}

extern "C" gn_status gn_mpnn_create(gn_mpnn** out, const float* init_params_host, void* stream) {
  using namespace gn;
  if (!out) return fail(GN_ERR_ARG, "gn_mpnn_create: out is NULL");
  *out = nullptr;
  if (!init_params_host) return fail(GN_ERR_ARG, "gn_mpnn_create: init_params is NULL");
  gn_mpnn* m = new gn_mpnn();
  struct Guard {
    gn_mpnn*& m;
    ~Guard() { if (m) gn_mpnn_destroy(m); }
  } guard{m};
  GN_CUDA(cudaGetDevice(&m->device));
  GN_CUDA(cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, m->device));
  GN_CUDA(cudaFuncSetAttribute((const void*)k_dense_fwd<kH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dense_fwd_smem<kH>()));
  GN_CUDA(cudaFuncSetAttribute((const void*)k_dense_fwd<kF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)dense_fwd_smem<kF>()));
  m->stream = (cudaStream_t)stream;
  const size_t nb = sizeof(float) * kNumParams;
  GN_CUDA(cudaMalloc(&m->d_w, nb));
  GN_CUDA(cudaMalloc(&m->d_wb, sizeof(__nv_bfloat16) * kNumParams));
  GN_CUDA(cudaMalloc(&m->d_g, nb));
  GN_CUDA(cudaMalloc(&m->d_m, nb));
  GN_CUDA(cudaMalloc(&m->d_v, nb));
  GN_CUDA(cudaMalloc(&m->d_loss, sizeof(double)));
  GN_CUDA(cudaMallocHost(&m->h_loss, sizeof(double)));
  GN_CUDA(cudaMemcpyAsync(m->d_w, init_params_host, nb, cudaMemcpyHostToDevice, m->stream));
  GN_CUDA(cudaMemsetAsync(m->d_g, 0, nb, m->stream));
  GN_CUDA(cudaMemsetAsync(m->d_m, 0, nb, m->stream));
  GN_CUDA(cudaMemsetAsync(m->d_v, 0, nb, m->stream));
  k_to_bf16<<<blk(kNumParams, 256), 256, 0, m->stream>>>(kNumParams, m->d_w, m->d_wb);
  GN_LAUNCHED();
  GN_CUDA(cudaStreamSynchronize(m->stream));
  *out = m;
  m = nullptr;
  return GN_OK;
}

extern "C" gn_status gn_mpnn_get_params(gn_mpnn* m, float* host_out) {
  using namespace gn;
  if (!m || !host_out) return fail(GN_ERR_ARG, "gn_mpnn_get_params: bad argument");
  GN_CUDA(cudaMemcpyAsync(host_out, m->d_w, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, m->stream));
  GN_CUDA(cudaStreamSynchronize(m->stream));
  return GN_OK;
}

extern "C" gn_status gn_mpnn_get_grads(gn_mpnn* m, float* host_out) {
  using namespace gn;
  if (!m || !host_out) return fail(GN_ERR_ARG, "gn_mpnn_get_grads: bad argument");
  GN_CUDA(cudaMemcpyAsync(host_out, m->d_g, sizeof(float) * kNumParams, cudaMemcpyDeviceToHost, m->stream));
  GN_CUDA(cudaStreamSynchronize(m->stream));
  return GN_OK;
}

// forward on graph g (its internal order); x0_out (caller order, device, may be NULL), target
// (caller order, device, NULL = inference only), *loss (host, may be NULL)
static gn_status mpnn_forward_impl(gn_mpnn* m, const gn_graph* g, float* x0_out, const float* target,
                                   double* loss, float alpha) {
  using namespace gn;
  if (!m || !g || !(alpha >= 0.0f && alpha <= 1.0f)) return fail(GN_ERR_ARG, "gn_mpnn_forward: bad argument");
  const int n = g->n;
  if (n == 0) return GN_OK;
  gn_status st = mpnn_reserve(m, n);
  if (st != GN_OK) return st;
  cudaStream_t s = m->stream;
  k_features<<<blk(n, 256), 256, 0, s>>>(n, g->d_row_ptr, g->d_col_idx, g->d_w, m->X);
  GN_LAUNCHED();
  const float* Hin = m->X;
  for (int l = 0; l < kL; ++l) {
    const __nv_bfloat16* Wb = m->d_wb + layer_off(l);
    // the dense layers: a grid of a few CTAs per SM walking the row tiles
    const int tiles = (n + kDenseRows - 1) / kDenseRows;
    float* Z = target ? m->Zs[l] : nullptr;  // pre-activations only for the backward
    if (l == 0) {
      k_aggregate<kF><<<blk(n, 256), 256, 0, s>>>(n, g->d_row_ptr, g->d_col_idx, Hin, m->Ms[l]);
      GN_LAUNCHED();
      k_dense_fwd<kF><<<std::min(tiles, 8 * m->num_sms), kDenseThreads, dense_fwd_smem<kF>(), s>>>(
          n, Hin, m->Ms[l], Wb, Z, m->Hs[l]);
      GN_LAUNCHED();
    } else {
      k_aggregate<kH><<<blk((int64_t)n * 32, 256), 256, 0, s>>>(n, g->d_row_ptr, g->d_col_idx, Hin, m->Ms[l]);
      GN_LAUNCHED();
      const int tc_tiles = (n + kTcRows - 1) / kTcRows;
      k_dense_fwd_tc<<<std::min(tc_tiles, 8 * m->num_sms), 32 * kTcWarps, 0, s>>>(n, Hin, m->Ms[l], Wb, Z,
                                                                                 m->Hs[l]);
      GN_LAUNCHED();
    }
    Hin = m->Hs[l];
  }
  if (target) {
    k_gather_caller<<<blk(n, 256), 256, 0, s>>>(n, target, g->d_perm, m->tgt);
    GN_LAUNCHED();
  }
  GN_CUDA(cudaMemsetAsync(m->d_loss, 0, sizeof(double), s));
  // the head reads targets in caller order through the permutation
  k_head<<<blk(n, kHeadRows), kHeadRows, 0, s>>>(n, m->Hs[kL - 1], m->d_wb + layer_off(kL), target, g->d_perm,
                                                 x0_out, m->dq, m->d_loss, g->d_row_ptr, alpha);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  m->n = n;
  m->last_graph = target ? g : nullptr;
  if (loss) {
    GN_CUDA(cudaMemcpyAsync(m->h_loss, m->d_loss, sizeof(double), cudaMemcpyDeviceToHost, s));
    GN_CUDA(cudaStreamSynchronize(s));
    *loss = *m->h_loss;
  }
  return GN_OK;
}

extern "C" gn_status gn_mpnn_forward(gn_mpnn* m, const gn_graph* g, float* x0_out, const float* target,
                                     double* loss) {
  return mpnn_forward_impl(m, g, x0_out, target, loss, 1.0f);
}

extern "C" gn_status gn_mpnn_predict(gn_mpnn* m, const gn_graph* g, float alpha, float* x0_out) {
  if (!x0_out) return gn::fail(GN_ERR_ARG, "gn_mpnn_predict: x0_out is NULL");
  gn_status st = mpnn_forward_impl(m, g, x0_out, nullptr, nullptr, alpha);
  if (st != GN_OK) return st;
  GN_CUDA(cudaStreamSynchronize(m->stream));
  return GN_OK;
}

// gradients of the last forward's loss, added into the gradient buffer
extern "C" gn_status gn_mpnn_backward(gn_mpnn* m, const gn_graph* g) {
  using namespace gn;
  if (!m || !g || m->last_graph != g) return fail(GN_ERR_ARG, "gn_mpnn_backward: needs a forward with targets on g");
  const int n = m->n;
  cudaStream_t s = m->stream;
  // three n x kH buffers rotate: cur = d loss / d H_l, dz = d loss / d Z_l, spare
  float* cur = m->bufA;
  float* dz = m->bufB;
  float* spare = m->bufC;
  k_head_bwd<<<blk(n, 256), 256, 0, s>>>(n, m->Hs[kL - 1], m->d_wb + layer_off(kL), m->dq, cur, m->part);
  GN_LAUNCHED();
  k_reduce_parts<<<blk(kH + 1, 256), 256, 0, s>>>((int)blk(n, 256), kH + 1, m->part, m->d_g + layer_off(kL));
  GN_LAUNCHED();
  const int rows_w = 256;
  for (int l = kL - 1; l >= 0; --l) {
    const __nv_bfloat16* Wb = m->d_wb + layer_off(l);
    float* dW = m->d_g + layer_off(l);
    const float* Hin = l == 0 ? m->X : m->Hs[l - 1];
    if (l == 0) {
      // the inputs are features: only dZ (for the weights) is needed
      k_dense_bwd_data<kF><<<blk(n, kRows), 256, 0, s>>>(n, cur, m->Zs[l], Wb, dz, spare, spare);
      GN_LAUNCHED();
      k_dense_bwd_weight<kF><<<blk(n, rows_w), 256, 0, s>>>(n, rows_w, dz, Hin, m->Ms[l], m->part);
      GN_LAUNCHED();
      k_reduce_parts<<<blk(2 * kH * kF + kH, 256), 256, 0, s>>>((int)blk(n, rows_w), 2 * kH * kF + kH, m->part, dW);
      GN_LAUNCHED();
    } else {
      // dZ -> dz; dH_in = dZ Ws -> spare; dM_in = dZ Wn -> cur (each CTA reads its rows of cur
      // into shared memory before writing them back)
      k_dense_bwd_data<kH><<<blk(n, kRows), 256, 0, s>>>(n, cur, m->Zs[l], Wb, dz, spare, cur);
      GN_LAUNCHED();
      k_dense_bwd_weight<kH><<<blk(n, rows_w), 256, 0, s>>>(n, rows_w, dz, Hin, m->Ms[l], m->part);
      GN_LAUNCHED();
      k_reduce_parts<<<blk(2 * kH * kH + kH, 256), 256, 0, s>>>((int)blk(n, rows_w), 2 * kH * kH + kH, m->part, dW);
      GN_LAUNCHED();
      // d loss / d H_{l-1} = dH_in + A^T (dM_in / deg)
      k_aggregate_t<kH><<<blk((int64_t)n * 32, 256), 256, 0, s>>>(n, g->d_row_ptr, g->d_col_idx, cur, spare);
      GN_LAUNCHED();
      std::swap(cur, spare);  // cur <- gradient of the previous layer's output
    }
  }
  GN_CUDA(cudaGetLastError());
  return GN_OK;
}

extern "C" gn_status gn_mpnn_zero_grad(gn_mpnn* m) {
  using namespace gn;
  if (!m) return fail(GN_ERR_ARG, "gn_mpnn_zero_grad: NULL");
  GN_CUDA(cudaMemsetAsync(m->d_g, 0, sizeof(float) * kNumParams, m->stream));
  return GN_OK;
}

// one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the accumulated gradients, then zero them
extern "C" gn_status gn_mpnn_step(gn_mpnn* m, float lr) {
  using namespace gn;
  if (!m || !(lr > 0.0f)) return fail(GN_ERR_ARG, "gn_mpnn_step: bad argument");
  m->adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - powf(b1, (float)m->adam_t), c2 = 1.0f - powf(b2, (float)m->adam_t);
  k_adam<<<blk(kNumParams, 256), 256, 0, m->stream>>>(kNumParams, m->d_w, m->d_g, m->d_m, m->d_v, m->d_wb, lr, b1,
                                                      b2, 1e-8f, c1, c2);
  GN_LAUNCHED();
  GN_CUDA(cudaMemsetAsync(m->d_g, 0, sizeof(float) * kNumParams, m->stream));
  GN_CUDA(cudaGetLastError());
  return GN_OK;
}
