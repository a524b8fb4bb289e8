// gn_extract.cu -- a8 of the path (gn_extract_is) and the FP64 diagnostics (gn_objective).
//
// Extraction (Sec. 2 independent sets; Sec. 6 "valid MIS after rounding"): S = {i : x_i > 1/2},
// an exact check of every edge for independence, a maximality check, the member list in
// ascending caller ids and W(S) in FP64.  All FP64 sums are two-pass, fixed order
// (per-CTA tree, then one CTA over the CTA partials), so they are deterministic.
#include <algorithm>
#include <cstring>

#include "gn_internal.cuh"

namespace gn {

static constexpr int kRedThreads = 256;
static constexpr int kRedBlocks = 1024;  // d_bsum holds 4 * kRedBlocks doubles

__device__ __forceinline__ double block_sum_d(double v, double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = dev::warp_sum_d(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += sh[j];
  __syncthreads();
  return t;  // valid in thread 0
}

// gather a caller-order vector into internal order
__global__ void k_gather(int n, const float* __restrict__ src, const int32_t* __restrict__ perm,
                         float* __restrict__ dst) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm[i]];
}

// objective and non-binary count of a state (internal order)
__global__ void k_stats(int n, const float* __restrict__ x, const float* __restrict__ w, double theta,
                        double* __restrict__ bsum) {
  __shared__ double sh[32];
  double o = 0.0, nb = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    o += (double)w[i] * (double)x[i];
    double xi = x[i];
    nb += (xi > theta && xi < 1.0 - theta) ? 1.0 : 0.0;
  }
  double to = block_sum_d(o, sh);
  double tn = block_sum_d(nb, sh);
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = to;
    bsum[kRedBlocks + blockIdx.x] = tn;
  }
}

// energy terms y_i ((y_i + gamma sum_j y_j)/2 - v_i), y = v x (Sec. 3), plus the objective, in
// FP64 with v = sqrt(w) from its float pair (v_hi + v_lo, about 2^-48 relative)
__global__ void k_energy(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                         const float* __restrict__ x, const float* __restrict__ v, const float* __restrict__ vlo,
                         const float* __restrict__ w, double gamma, double* __restrict__ bsum) {
  __shared__ double sh[32];
  double en = 0.0, o = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = rp[i]; k < rp[i + 1]; ++k) {
      int j = ci[k];
      s += ((double)v[j] + (double)vlo[j]) * (double)x[j];
    }
    const double vi = (double)v[i] + (double)vlo[i];
    double yi = vi * (double)x[i];
    en += yi * (0.5 * (yi + gamma * s) - vi);
    o += (double)w[i] * (double)x[i];
  }
  double te = block_sum_d(en, sh);
  double to = block_sum_d(o, sh);
  if (threadIdx.x == 0) {
    bsum[blockIdx.x] = to;
    bsum[kRedBlocks + blockIdx.x] = te;
  }
}

// fixed-order sum of nparts CTA partials for `lanes` quantities
__global__ void k_finish(const double* __restrict__ bsum, int nparts, int lanes, double* __restrict__ out) {
  __shared__ double sh[32];
  for (int q = 0; q < lanes; ++q) {
    double t = 0.0;
    for (int j = threadIdx.x; j < nparts; j += blockDim.x) t += bsum[q * kRedBlocks + j];
    double tt = block_sum_d(t, sh);
    if (threadIdx.x == 0) out[q] = tt;
  }
}

// rounding (internal order) and the exact independence / maximality checks per row
__global__ void k_round(int n, const float* __restrict__ x, uint8_t* __restrict__ mask) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) mask[i] = x[i] > 0.5f ? 1 : 0;
}

__global__ void k_check_is(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                           const uint8_t* __restrict__ mask, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const bool in = mask[i] != 0;
  bool covered = false;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    if (mask[ci[k]]) {
      if (in) { atomicOr(&flags[0], 1); return; }  // edge inside S
      covered = true;
      break;
    }
  }
  if (!in && !covered) atomicOr(&flags[1], 1);      // not maximal
}

// caller-order membership, per-CTA member counts and W(S) partials
__global__ void k_members_count(int n, const uint8_t* __restrict__ mask_int,
                                const int32_t* __restrict__ iperm, const float* __restrict__ w_int,
                                uint8_t* __restrict__ mask_c, int* __restrict__ bcount,
                                double* __restrict__ bsum) {
  __shared__ double sh[32];
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  double wsum = 0.0;
  if (c < n) {
    int i = iperm ? iperm[c] : c;
    uint8_t m = mask_int[i];
    mask_c[c] = m;
    if (m) {
      atomicAdd(&cnt, 1);
      wsum = (double)w_int[i];
    }
  }
  double t = block_sum_d(wsum, sh);
  if (threadIdx.x == 0) {
    bcount[blockIdx.x] = cnt;
    bsum[blockIdx.x] = t;
  }
}

// exclusive scan of the per-CTA counts (one CTA, sequential per thread chunk) + W(S) total
// exclusive prefix of the per-block member counts (in place) and their total, and the total
// weight (FP64 sum of the per-block partials).  One CTA: each thread takes a contiguous chunk,
// then a block scan of the chunk counts (the FP64 adds run in parallel, not as one chain).
__global__ void __launch_bounds__(1024) k_scan_counts(int nb, int* __restrict__ bcount, int* __restrict__ total,
                                                      const double* __restrict__ bsum,
                                                      double* __restrict__ wtotal) {
  __shared__ int s_warp[32];
  __shared__ double sh[32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
  const int C = (nb + blockDim.x - 1) / blockDim.x;
  const int a = min(nb, t * C), b = min(nb, a + C);
  int cnt = 0;
  double ws = 0.0;
  for (int j = a; j < b; ++j) {
    cnt += bcount[j];
    ws += bsum[j];
  }
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < nwarps ? s_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    s_warp[lane] = v;  // inclusive totals of warps 0..lane
  }
  __syncthreads();
  int run = incl - cnt + (warp > 0 ? s_warp[warp - 1] : 0);
  for (int j = a; j < b; ++j) {
    const int c = bcount[j];
    bcount[j] = run;
    run += c;
  }
  if (t == (int)blockDim.x - 1) *total = run;
  const double tw = block_sum_d(ws, sh);
  if (t == 0) *wtotal = tw;
}

__global__ void k_members_write(int n, const uint8_t* __restrict__ mask_c, const int* __restrict__ boff,
                                int32_t* __restrict__ members) {
  __shared__ int warp_cnt[32];
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool m = c < n && mask_c[c];
  unsigned bal = __ballot_sync(0xffffffffu, m);
  if (lane == 0) warp_cnt[warp] = __popc(bal);
  __syncthreads();
  int off = boff[blockIdx.x];
  for (int j = 0; j < warp; ++j) off += warp_cnt[j];
  if (m) members[off + __popc(bal & ((1u << lane) - 1u))] = c;
}

gn_status to_internal(gn_graph* g, const float* x_caller, const float** x_int) {
  if (!x_caller) {
    if (!g->has_state) return fail(GN_ERR_ARG, "no state: pass x or call gn_run first");
    *x_int = g->d_x;
    return GN_OK;
  }
  const float* dev = nullptr;
  gn_status st = upload_or_alias(g, x_caller, sizeof(float) * g->n, (const void**)&dev);
  if (st != GN_OK) return st;
  if (g->d_perm) {
    k_gather<<<(g->n + 255) / 256, 256, 0, g->stream>>>(g->n, dev, g->d_perm, g->d_tmp);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
    *x_int = g->d_tmp;
  } else {
    *x_int = dev;
  }
  return GN_OK;
}

static int red_blocks(int n) { return std::min(kRedBlocks, std::max(1, (n + kRedThreads - 1) / kRedThreads)); }

gn_status state_stats(gn_graph* g, const float* x_int, double theta, double* obj, unsigned* nonbin) {
  const int nb = red_blocks(g->n);
  k_stats<<<nb, kRedThreads, 0, g->stream>>>(g->n, x_int, g->d_w, theta, g->d_bsum);
  GN_LAUNCHED();
  k_finish<<<1, kRedThreads, 0, g->stream>>>(g->d_bsum, nb, 2, g->d_red);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  GN_CUDA(cudaMemcpyAsync(g->h_red, g->d_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  *obj = g->h_red[0];
  *nonbin = (unsigned)g->h_red[1];
  return GN_OK;
}

}  // namespace gn

extern "C" gn_status gn_objective(gn_graph* g, const float* x, double gamma, double* obj, double* energy) {
  using namespace gn;
  if (!g || !std::isfinite(gamma)) return fail(GN_ERR_ARG, "gn_objective: bad argument");
  GN_CUDA(cudaSetDevice(g->device));
  if (g->n == 0) {
    if (obj) *obj = 0.0;
    if (energy) *energy = 0.0;
    return GN_OK;
  }
  const float* xi = nullptr;
  gn_status st = to_internal(g, x, &xi);
  if (st != GN_OK) return st;
  const int nb = red_blocks(g->n);
  k_energy<<<nb, kRedThreads, 0, g->stream>>>(g->n, g->d_row_ptr, g->d_col_idx, xi, g->d_v, g->d_vlo,
                                              g->d_w, gamma, g->d_bsum);
  GN_LAUNCHED();
  k_finish<<<1, kRedThreads, 0, g->stream>>>(g->d_bsum, nb, 2, g->d_red);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  GN_CUDA(cudaMemcpyAsync(g->h_red, g->d_red, sizeof(double) * 2, cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (obj) *obj = g->h_red[0];
  if (energy) *energy = g->h_red[1];
  return GN_OK;
}

extern "C" gn_status gn_extract_is(gn_graph* g, const float* x, uint8_t* mask, int32_t* members,
                                   int32_t* count, double* weight) {
  using namespace gn;
  if (!g) return fail(GN_ERR_ARG, "gn_extract_is: NULL handle");
  GN_CUDA(cudaSetDevice(g->device));
  const int n = g->n;
  if (n == 0) {
    if (count) *count = 0;
    if (weight) *weight = 0.0;
    return GN_OK;
  }
  const float* xi = nullptr;
  gn_status st = to_internal(g, x, &xi);
  if (st != GN_OK) return st;
  const int T = 256;
  const int nbk = (n + T - 1) / T;
  int* ctot = &g->d_flags[4];
  int* flags = g->d_flags;
  GN_CUDA(cudaMemsetAsync(g->d_flags, 0, sizeof(int) * 8, g->stream));
  k_round<<<nbk, T, 0, g->stream>>>(n, xi, g->d_mask);
  GN_LAUNCHED();
  k_check_is<<<nbk, T, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, g->d_mask, flags);
  GN_LAUNCHED();
  k_members_count<<<nbk, T, 0, g->stream>>>(n, g->d_mask, g->d_iperm, g->d_w, g->d_mask_c,
                                            g->d_bcount, g->d_bws);
  GN_LAUNCHED();
  k_scan_counts<<<1, 1024, 0, g->stream>>>(nbk, g->d_bcount, ctot, g->d_bws, g->d_red);
  GN_LAUNCHED();
  k_members_write<<<nbk, T, 0, g->stream>>>(n, g->d_mask_c, g->d_bcount, g->d_members);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  GN_CUDA(cudaMemcpyAsync(g->h_flags, g->d_flags, sizeof(int) * 8, cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaMemcpyAsync(g->h_red, g->d_red, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  const int cnt = g->h_flags[4];
  if (mask) {
    st = copy_out(g, mask, g->d_mask_c, (size_t)n);
    if (st != GN_OK) return st;
  }
  if (members) {
    st = copy_out(g, members, g->d_members, sizeof(int32_t) * (size_t)cnt);
    if (st != GN_OK) return st;
  }
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (count) *count = cnt;
  if (weight) *weight = g->h_red[0];
  if (g->h_flags[0]) return fail(GN_ERR_NOT_INDEPENDENT, "gn_extract_is: the rounded set has an edge inside");
  if (g->h_flags[1]) return fail(GN_WARN_NOT_MAXIMAL, "gn_extract_is: the rounded set is not maximal");
  return GN_OK;
}
