// gn_iterate.cu -- a2..a7 of the path: the persistent fused WRGN kernel and gn_run.
//
// One cooperative launch runs every iteration of a gn_run call.  Each CTA owns a
// contiguous range of (internal) rows, balanced by entries + rows, and keeps its rows'
// v, y, x and (when it fits) its slice of col_idx in shared memory for the whole run.
// Per iteration k (App. B, weighted state y = v (.) x, B = I + gamma_k A):
//   gather   s_i = sum_{j in N(i)} y_j      (G lanes per light row, a warp per heavy row)
//   update   d_i = y_i + gamma_k s_i = (B y)_i;  x_i' = y_i / d_i,  y_i' = v_i x_i'
//            (d_i <= 1e-9: x_i' = 1/2, the safe division of the appendix module)
//   check    every c iterations: max |x'-x| and the non-binary count (the stop test) plus
//            FP64 sums of |x'-x|, w x' (Thm. 3) and y (d/2 - v) (= E~(y), Sec. 3)
//   barrier  a bounded grid barrier; at a check every CTA then reduces the same per-CTA
//            partials in the same order, so all CTAs take the same stop decision.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "gn_internal.cuh"
#include "gn_iter_common.cuh"

namespace gn {

// Gather modes of the persistent kernel
enum GatherMode : int {
  MODE_GMEM = 0,       // neighbour ids read from global memory, values gathered from L1/L2
  MODE_SMEM_CSR = 1,   // the CTA's neighbour ids held in shared memory, values from L1/L2
  MODE_HALO = 2,       // gn_halo.cu: external halo values staged in shared memory
};

gn_status build_halo(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                     const std::vector<int32_t>& part, size_t smem_limit, int want, bool* fits);  // gn_halo.cu
const void* halo_kernel(int rows_pad, bool push, bool tagged);

// The generic persistent kernel: values gathered through L1/L2 (MODE_GMEM, MODE_SMEM_CSR),
// G lanes per light row and a warp per heavy row.
template <int G, bool SMEM_CSR>
__global__ void __launch_bounds__(kThreads, 1) k_gn_persistent(const IterParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TailShared T;
  __shared__ int s_nheavy;
  const int R = P.rows_pad;
  RowArrays S;
  S.sum = reinterpret_cast<float*>(smem);
  S.yh = S.sum + R;
  S.yl = S.yh + R;
  S.x = S.yl + R;
  S.vh = S.x + R;
  S.vl = S.vh + R;
  int* s_rp = reinterpret_cast<int*>(S.vl + R);
  int* s_heavy = s_rp + R + 4;
  int* s_ci = s_heavy + R;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int b = blockIdx.x;
  const int rb = P.part[b], nr = P.part[b + 1] - rb;
  const int e0 = P.row_ptr[rb];

  // a failed start-state validation (written before the launch) ends the run at once
  if (dev::ld_relaxed_int(P.status) != 0) return;

  if (tid == 0) s_nheavy = 0;
  for (int i = tid; i <= nr; i += blockDim.x) s_rp[i] = P.row_ptr[rb + i] - e0;
  for (int i = tid; i < nr; i += blockDim.x) {
    S.vh[i] = P.v[rb + i];
    S.vl[i] = P.vlo[rb + i];
    const Own o = own_load(P.y0[rb + i], P.ylo[rb + i], P.x[rb + i], P.yexp[rb + i]);
    S.yh[i] = o.pub;
    S.yl[i] = o.aux;
    S.x[i] = o.xs;
  }
  __syncthreads();
  if (SMEM_CSR) {
    const int ne = s_rp[nr];
    for (int e = tid; e < ne; e += blockDim.x) s_ci[e] = P.col_idx[e0 + e];
  }
  for (int i = tid; i < nr; i += blockDim.x)
    if (s_rp[i + 1] - s_rp[i] > P.heavy) s_heavy[atomicAdd(&s_nheavy, 1)] = i;
  set_gamma(P, P.k_start, T);
  __syncthreads();
  const int* __restrict__ ci = SMEM_CSR ? s_ci : (P.col_idx + e0);
  const int nheavy = s_nheavy;
  const float th_lo = (float)P.theta, th_hi = (float)(1.0 - P.theta);

  unsigned hits = 0;
  int parity = 0, slot = 0, stop = 0;
  unsigned nbar = 0;
  int nchk = 0;  // checks so far (selects the check word)
  int k = P.k_start;
  const int grp = tid / G, gl = tid & (G - 1), ngrp = blockDim.x / G;
  int next_chk = (P.k_start / P.check_every + 1) * P.check_every;  // a check follows step next_chk - 1

  for (; k < P.k_end; ++k) {
    const dev::f2 gam = {T.gh, T.gl};
    const float2 gnext = gamma_fetch(P, k + 1);
    const float* __restrict__ yin = parity ? P.y1 : P.y0;
    float* __restrict__ yout = parity ? P.y0 : P.y1;

    // ---- gather: light rows, G lanes per row
    for (int base = 0; base < nr; base += ngrp) {
      const int r = base + grp;
      float acc = 0.0f;
      bool mine = false;
      if (r < nr) {
        const int a = s_rp[r], c = s_rp[r + 1];
        if (c - a <= P.heavy) {
          mine = true;
          for (int e = a + gl; e < c; e += G) acc += yin[ci[e]];
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (mine && gl == 0) S.sum[r] = acc;
    }
    // ---- gather: heavy rows, a warp per row
    for (int h = warp; h < nheavy; h += nwarps) {
      const int r = s_heavy[h];
      const int a = s_rp[r], c = s_rp[r + 1];
      float acc = 0.0f;
      for (int e = a + lane; e < c; e += 32) acc += yin[ci[e]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) S.sum[r] = acc;
    }
    __syncthreads();

    // ---- update, stop-test partials, barrier, stop decision
    const bool due = k + 1 == next_chk;
    const bool check = due || (k + 1 == P.k_end);
    if (due) next_chk += P.check_every;
    CheckAcc acc;
    update_rows(S, nr, rb, P.w, yout, gam, check, th_lo, th_hi, hits, acc);
    gamma_store(gnext, T);  // visible to every thread after the barrier's __syncthreads
    stop = check ? check_barrier(P, false, false, nbar, nchk, gam, k, acc, T)
                 : barrier_and_stop(P, false, false, nbar, slot, false, gam, k, T);
    if (stop == 2) break;
    parity ^= 1;
    if (stop) {
      ++k;
      break;
    }
  }
  if (stop == 2) return;  // timeout: the status word says so; leave the state as is
  finish_run(P, S, rb, nr, hits, k, parity, T);
}

// gamma_k of Sec. 6 for k < len, in FP64 (the paper's ramp formula), split into float pairs
__global__ void k_gamma_table(int len, int mode, double g0, double g1, int T, float2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  const dev::f2 p = dev::split_f64(dev::gamma_at(mode, g0, g1, T, k));
  out[k] = make_float2(p.hi, p.lo);
}

// ------------------------------------------------------------------------------------------
// start state: x0 (caller order, or 1/(deg+1)), validation (Def. 1), y0 = v (.) x0

__global__ void k_init_state(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             const float* __restrict__ v, const float* __restrict__ vlo,
                             const float* __restrict__ x0, const int32_t* __restrict__ perm,
                             float* __restrict__ x, float* __restrict__ y, float* __restrict__ ylo,
                             float* __restrict__ yexp, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = rp[i], e = rp[i + 1];
  float xi;
  if (x0) {
    xi = x0[perm ? perm[i] : i];
  } else {
    xi = __frcp_rn((float)(e - b + 1));
  }
  bool bad = !(xi >= 0.0f) || !isfinite(xi);
  if (x0 && !bad && !(xi > 0.0f)) {
    // (A + I) x0 > 0: a zero needs a positive neighbour
    bool pos = false;
    for (int k = b; k < e && !pos; ++k) pos = x0[perm ? perm[ci[k]] : ci[k]] > 0.0f;
    bad = !pos;
  }
  if (bad) atomicOr(status, DEV_NOT_NORMALIZABLE);
  x[i] = xi;
  dev::f2 yy = dev::mul_f2(dev::f2{v[i], vlo[i]}, dev::f2{xi, 0.0f});
  y[i] = yy.hi;
  ylo[i] = yy.lo;
  yexp[i] = 0.0f;
}

__global__ void k_to_caller(int n, const float* __restrict__ x_int, const int32_t* __restrict__ iperm,
                            float* __restrict__ out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float xv = x_int[iperm ? iperm[i] : i];
  out[i] = fminf(fmaxf(xv, 0.0f), 1.0f);
}

// ------------------------------------------------------------------------------------------

using KernelFn = void (*)(const IterParams);

static KernelFn pick_kernel(int G, int mode) {
  const bool sm = mode == MODE_SMEM_CSR;
#define GN_PICK(g) \
  case g:          \
    return sm ? (KernelFn)k_gn_persistent<g, true> : (KernelFn)k_gn_persistent<g, false>;
  switch (G) {
    GN_PICK(1)
    GN_PICK(2)
    GN_PICK(4)
    GN_PICK(8)
    GN_PICK(16)
    GN_PICK(32)
  }
#undef GN_PICK
  return nullptr;
}

static constexpr size_t kSmemLimit = 220 * 1024;
static constexpr int64_t kHeavyRowCost = 64;  // the halo mode's heavy-row threshold

gn_status configure_partition(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci) {
  const int n = g->n;
  const int64_t nnz = g->nnz;
  // Per-row cost in entry units: its entries, plus alpha for the row bookkeeping and update.
  // Entries of rows above kHeavyRowCost entries count twice: they are summed by whole warps
  // from randomly placed neighbours (no bank-aware layout), at about half the rate.
  const int64_t alpha = 4;
  auto cost = [&](int i) {
    const int64_t d = rp[i + 1] - rp[i];
    return d + (d > kHeavyRowCost ? d : 0) + alpha;
  };
  // the prefix C in two passes over the same row blocks on the host threads: each block's sum,
  // then each block's prefix from its offset
  std::unique_ptr<int64_t[]> C(new int64_t[(size_t)n + 1]);
  std::vector<int64_t> boff(host_threads() + 1, 0);
  constexpr int kRowGrain = 16384;
  parallel_for(n, kRowGrain, [&](int lo, int hi, int t) {
    int64_t sum = 0;
    for (int i = lo; i < hi; ++i) sum += cost(i);
    boff[t + 1] = sum;
  });
  for (size_t t = 1; t < boff.size(); ++t) boff[t] += boff[t - 1];
  C[0] = 0;
  parallel_for(n, kRowGrain, [&](int lo, int hi, int t) {
    int64_t at = boff[t];
    for (int i = lo; i < hi; ++i) C[i + 1] = at += cost(i);
  });
  const int64_t total = C[n];
  (void)nnz;
  int nb = (int)std::min<int64_t>(g->num_sms, std::max<int64_t>(1, (total + 2047) / 2048));
  // balanced contiguous split of the prefix cost C
  std::vector<int32_t> part(nb + 1);
  part[0] = 0;
  for (int b = 1; b < nb; ++b) {
    const int64_t want = total * b / nb;
    int lo = part[b - 1], hi = n;  // smallest i with C(i) >= want
    while (lo < hi) {
      int mid = lo + (hi - lo) / 2;
      if (C[mid] >= want) hi = mid; else lo = mid + 1;
    }
    part[b] = lo;
  }
  part[nb] = n;
  int max_rows = 0;
  int64_t max_ents = 0;
  for (int b = 0; b < nb; ++b) {
    max_rows = std::max(max_rows, part[b + 1] - part[b]);
    max_ents = std::max<int64_t>(max_ents, (int64_t)rp[part[b + 1]] - rp[part[b]]);
  }
  const double avg = n > 0 ? (double)nnz / n : 0.0;
  int G = 1;
  while (G < 32 && G * 3 < avg) G <<= 1;
  g->group = G;
  g->heavy = 16 * G;
  g->nblocks = nb;
  g->max_rows = max_rows;
  g->max_ents = max_ents;
  const int R = (max_rows + 3) & ~3;
  const size_t rows_bytes = sizeof(float) * 6 * (size_t)R + sizeof(int) * ((size_t)R + 4) + sizeof(int) * (size_t)R;

  const size_t csr_s = rows_bytes + 4 * (size_t)max_ents;
  const int want = g->gather;
  bool halo_fits = false;
  const bool want_halo = want == GN_GATHER_HALO || want == GN_GATHER_HALO_PULL || want == GN_GATHER_HALO_PUSH;
  if (want == GN_GATHER_AUTO || want_halo) {
    gn_status hst = build_halo(g, rp, ci, part, kSmemLimit, want == GN_GATHER_AUTO ? GN_GATHER_HALO : want,
                               &halo_fits);
    if (hst != GN_OK) return hst;
    if (want_halo && !halo_fits)
      return fail(GN_ERR_TOO_LARGE, "gn_create: the halo gather mode does not fit shared memory");
  }
  KernelFn fn = nullptr;
  int per_sm = 0;
  if (halo_fits) {
    g->mode = MODE_HALO;
    g->gather = GN_GATHER_HALO;
    const void* hk = halo_kernel(g->rows_pad_halo, g->halo_push, false);
    const void* hkt = halo_kernel(g->rows_pad_halo, g->halo_push, true);
    GN_CUDA(cudaFuncSetAttribute(hk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    GN_CUDA(cudaFuncSetAttribute(hkt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
    int per_sm_t = 0;
    GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (KernelFn)hk, kThreads, g->smem_bytes));
    GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_t, (KernelFn)hkt, kThreads, g->smem_bytes));
    per_sm = std::min(per_sm, per_sm_t);
  } else {
    if (want == GN_GATHER_SMEM_CSR && csr_s > kSmemLimit)
      return fail(GN_ERR_TOO_LARGE, "gn_create: the CSR-in-shared-memory mode does not fit");
    if (want != GN_GATHER_GLOBAL && csr_s <= kSmemLimit) {
      g->mode = MODE_SMEM_CSR;
      g->gather = GN_GATHER_SMEM_CSR;
      g->smem_bytes = csr_s;
    } else if (rows_bytes <= kSmemLimit) {
      g->mode = MODE_GMEM;
      g->gather = GN_GATHER_GLOBAL;
      g->smem_bytes = rows_bytes;
    } else {
      return fail(GN_ERR_TOO_LARGE, "gn_create: a CTA's rows exceed shared memory (graph too large)");
    }
    fn = pick_kernel(G, g->mode);
    // the attribute is an upper bound shared by every graph that uses this instance
    GN_CUDA(cudaFuncSetAttribute((const void*)fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kSmemLimit));
    GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, g->smem_bytes));
  }
  g->csr_in_smem = g->mode != MODE_GMEM;
  g->threads = kThreads;
  if (per_sm < 1 || nb > per_sm * g->num_sms)
    return fail(GN_ERR_TOO_LARGE, "gn_create: persistent kernel does not fit co-resident");
  GN_CUDA(cudaMalloc(&g->d_part, sizeof(int32_t) * (nb + 1)));
  GN_CUDA(cudaMemcpyAsync(g->d_part, part.data(), sizeof(int32_t) * (nb + 1), cudaMemcpyHostToDevice,
                          g->stream));
  GN_CUDA(cudaMalloc(&g->d_partials, sizeof(CheckPartial) * 2 * nb));
  GN_CUDA(cudaMalloc(&g->d_iterflag, sizeof(unsigned) * dev::kFlagStride * nb));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  return GN_OK;
}

gn_status record_forward(gn_graph* g, int k_start, int k_end, const gn_params& p, DevInfo* out, float* ms);  // gn_adjoint.cu

// gamma_k on the host, same arithmetic as the device (host code is built without FMA
// contraction)
double host_gamma(const gn_params& p, int k) {
  if (p.gamma_mode == GN_GAMMA_FIXED || p.ramp_iters <= 1) return p.gamma1;
  int kk = k < p.ramp_iters - 1 ? k : p.ramp_iters - 1;
  double t = (double)kk / (double)(p.ramp_iters - 1);
  return t * p.gamma1 + (1.0 - t) * p.gamma0;
}

gn_status init_state(gn_graph* g, const float* x0_dev) {
  if (g->n == 0) return GN_OK;
  k_init_state<<<(g->n + 255) / 256, 256, 0, g->stream>>>(g->n, g->d_row_ptr, g->d_col_idx, g->d_v,
                                                           g->d_vlo, x0_dev, g->d_perm, g->d_x,
                                                           g->d_y[0], g->d_ylo, g->d_yexp,
                                                           &g->d_info->status);
  g->state_parity = 0;
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  return GN_OK;
}

// The stop test's thresholds for the device (which does it without FP64): gamma (1 - theta) >
// theta <=> gamma > theta / (1 - theta) (theta < 1/2), that threshold as a float pair; the
// residual test r <= tol for an FP32 r <=> r <= the largest float <= tol.
void set_stop_thresholds(IterParams& P, double theta, double tol) {
  P.theta = theta;
  P.tol = tol;
  const double thr = theta / (1.0 - theta);
  P.thr_hi = (float)thr;
  P.thr_lo = (float)(thr - (double)P.thr_hi);
  P.res_test = tol >= 0.0 ? 1 : 0;
  float f = (float)tol;
  if ((double)f > tol) f = std::nextafter(f, -INFINITY);
  P.tol_f = f;
}

// Runs iterations k_start..k_end-1 from d_y[parity0] / d_x; the caller has zeroed d_info
// except for a start-state status.  Fills *out from the device summary.
gn_status run_iterations(gn_graph* g, int k_start, int k_end, double tol, const gn_params& p,
                         int parity0, DevInfo* out, float* ms, int* kernel_used) {
  IterParams P;
  P.row_ptr = g->d_row_ptr;
  P.col_idx = g->d_col_idx;
  P.v = g->d_v;
  P.vlo = g->d_vlo;
  P.w = g->d_w;
  P.part = g->d_part;
  P.y0 = g->d_y[parity0];
  P.y1 = g->d_y[parity0 ^ 1];
  P.x = g->d_x;
  P.ylo = g->d_ylo;
  P.yexp = g->d_yexp;
  P.hoff = g->d_hoff;
  P.hblob = g->d_hblob;
  P.halo_pad = g->halo_pad;
  P.partials = g->d_partials;
  P.bar = g->d_bar;
  P.status = &g->d_info->status;
  P.info = g->d_info;
  P.n = g->n;
  P.nblocks = g->nblocks;
  P.k_start = k_start;
  P.k_end = k_end;
  P.gamma_mode = p.gamma_mode;
  P.gamma0 = p.gamma0;
  P.gamma1 = p.gamma1;
  P.ramp = p.ramp_iters;
  P.check_every = p.check_every;
  set_stop_thresholds(P, p.theta_bin, tol);
  P.heavy = g->heavy;
  P.rows_pad = g->mode == MODE_HALO ? g->rows_pad_halo : ((g->max_rows + 3) & ~3);
  P.spin_limit = p.spin_limit > 0 ? p.spin_limit : (1ll << 22);
  const bool tagged = g->mode == MODE_HALO && (p.sync == GN_SYNC_TAGGED || p.sync == GN_SYNC_AUTO);
  P.unreachable = p.debug_unreachable_barrier != 0 && !(tagged && p.debug_unreachable_barrier == 2) ? 1 : 0;
  P.bad_tag = tagged && p.debug_unreachable_barrier == 2 ? 1 : 0;
  P.iterflag = (g->mode == MODE_HALO && p.sync == GN_SYNC_NEIGHBOUR) ? g->d_iterflag : nullptr;
  P.inbox = g->d_inbox;
  P.inbox_len = g->inbox_len;
  // gamma table: one entry per iteration up to the end of the ramp (gamma is constant after)
  const int glen = (p.gamma_mode == GN_GAMMA_FIXED || p.ramp_iters <= 1)
                       ? 1
                       : std::max(1, std::min(k_end, p.ramp_iters));
  if (glen > g->gtab_cap) {
    if (g->d_gtab) cudaFree(g->d_gtab);
    g->d_gtab = nullptr;
    g->gtab_cap = 0;
    GN_CUDA(cudaMalloc(&g->d_gtab, sizeof(float2) * glen));
    g->gtab_cap = glen;
  }
  k_gamma_table<<<(glen + 255) / 256, 256, 0, g->stream>>>(glen, p.gamma_mode, p.gamma0, p.gamma1,
                                                           p.ramp_iters, (float2*)g->d_gtab);
  GN_LAUNCHED();
  P.gtab = (const float2*)g->d_gtab;
  P.gtab_len = glen;
  KernelFn fn = g->mode == MODE_HALO ? (KernelFn)halo_kernel(g->rows_pad_halo, g->halo_push, tagged)
                                     : pick_kernel(g->group, g->mode);
  GN_CUDA(cudaMemsetAsync(g->d_bar, 0, sizeof(unsigned) * 8, g->stream));  // counter and check words
  if (P.iterflag)
    GN_CUDA(cudaMemsetAsync(g->d_iterflag, 0, sizeof(unsigned) * dev::kFlagStride * g->nblocks, g->stream));
  void* args[] = {(void*)&P};
  GN_CUDA(cudaEventRecord(g->ev0, g->stream));
  GN_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(g->nblocks), dim3(g->threads), args,
                                      g->smem_bytes, g->stream));
  GN_LAUNCHED();
  GN_CUDA(cudaEventRecord(g->ev1, g->stream));
  GN_CUDA(cudaMemcpyAsync(out, g->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (ms) GN_CUDA(cudaEventElapsedTime(ms, g->ev0, g->ev1));
  if (kernel_used) *kernel_used = GN_KERNEL_PERSISTENT;
  return GN_OK;
}

// GN_KERNEL_CTA: the whole run in one CTA, through a one-instance batch over the handle's CSR
// (internal order, device-resident; built on first use).  The start state is d_x (written by
// init_state) and the result goes back there.
static gn_status run_cta(gn_graph* g, int max_iters, double tol, const gn_params& p, DevInfo* out, float* ms) {
  if (!g->cta) {
    const int64_t off[4] = {0, (int64_t)g->n, 0, g->nnz};
    GN_CUDA(cudaMalloc(&g->d_cta_off, sizeof off));
    GN_CUDA(cudaMemcpyAsync(g->d_cta_off, off, sizeof off, cudaMemcpyHostToDevice, g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
    gn_status st = gn_batch_create(&g->cta, 1, g->d_cta_off, g->d_cta_off + 2, g->d_row_ptr, g->d_col_idx,
                                   g->d_w, nullptr, GN_DEVICE, g->stream);
    if (st != GN_OK) {
      g->cta = nullptr;
      return st;
    }
  }
  gn_batch_info bi;
  gn_status st = gn_batch_run(g->cta, g->d_x, max_iters, tol, &p, g->d_x, &bi);
  if (st < 0) return st;
  memset(out, 0, sizeof *out);
  out->iters = bi.iters;
  out->converged = bi.converged;
  out->binary = bi.binary;
  out->nonbin = bi.binary ? 0u : 1u;  // the batch reports binarity, not the count
  out->resid_inf = bi.resid_inf;
  out->resid_l1 = bi.resid_l1;
  out->objective = bi.objective;
  out->energy = bi.energy;
  out->hits = (unsigned long long)bi.safe_div_hits;
  *ms = gn_batch_last_ms(g->cta);
  return GN_OK;
}

}  // namespace gn

// ------------------------------------------------------------------------------------------

extern "C" gn_status gn_run(gn_graph* g, const float* x0, int max_iters, double tol,
                            const gn_params* pin, int start_iter, float* x_out, gn_run_info* info) {
  using namespace gn;
  if (!g) return fail(GN_ERR_ARG, "gn_run: NULL handle");
  gn_params p;
  if (pin) p = *pin; else gn_default_params(&p);
  if (start_iter < 0 || max_iters < start_iter || p.check_every < 1 || !(p.theta_bin < 0.5) ||
      !std::isfinite(p.gamma0) || !std::isfinite(p.gamma1) || p.gamma1 < 0 || p.gamma0 < 0 ||
      (p.gamma_mode != GN_GAMMA_PURSUIT && p.gamma_mode != GN_GAMMA_FIXED) ||
      p.kernel < GN_KERNEL_AUTO || p.kernel > GN_KERNEL_CTA || p.sync < GN_SYNC_AUTO ||
      p.sync > GN_SYNC_TAGGED)
    return fail(GN_ERR_ARG, "gn_run: bad argument");
  GN_CUDA(cudaSetDevice(g->device));
  GN_CUDA(cudaMemsetAsync(g->d_info, 0, sizeof(DevInfo), g->stream));
  gn_status st = GN_OK;
  if (p.kernel == GN_KERNEL_CTA && (p.resume || p.record || start_iter != 0))
    return fail(GN_ERR_ARG, "gn_run: the CTA kernel runs whole runs (start_iter 0, no record or resume)");
  if (p.resume) {
    if (!g->has_state) return fail(GN_ERR_ARG, "gn_run: resume without a previous run on this handle");
    if (g->state_cta) return fail(GN_ERR_ARG, "gn_run: the last run used the CTA kernel and cannot be resumed");
  } else {
    const float* x0_dev = nullptr;
    if (x0) {
      st = upload_or_alias(g, x0, sizeof(float) * g->n, (const void**)&x0_dev);
      if (st != GN_OK) return st;
    }
    st = init_state(g, x0_dev);
    if (st != GN_OK) return st;
  }
  const int parity0 = g->state_parity;

  DevInfo di;
  memset(&di, 0, sizeof di);
  float ms = 0.0f;
  int kused = GN_KERNEL_PERSISTENT;
  if ((int64_t)(max_iters - start_iter) * g->nblocks >= (int64_t)1 << 31)
    return fail(GN_ERR_TOO_LARGE, "gn_run: too many iterations for one call; split the run with start_iter");
  if (p.record && max_iters > start_iter && g->n > 0) {
    // differentiable form: exactly max_iters - start_iter steps with sqrt(T) checkpoints
    if (p.resume) return fail(GN_ERR_ARG, "gn_run: record and resume cannot be combined");
    GN_CUDA(cudaMemcpyAsync(&di, g->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
    if (di.status == 0) {
      st = record_forward(g, start_iter, max_iters, p, &di, &ms);
      if (st != GN_OK) return st;
      st = state_stats(g, g->d_x, p.theta_bin, &di.objective, &di.nonbin);
      if (st != GN_OK) return st;
      di.binary = di.nonbin == 0;
      di.converged = di.binary && host_gamma(p, max_iters - 1) * (1.0 - p.theta_bin) > p.theta_bin;
    }
  } else if (max_iters > start_iter && g->n > 0 && p.kernel == GN_KERNEL_CTA) {
    GN_CUDA(cudaMemcpyAsync(&di, g->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
    if (di.status == 0) {  // the start state passed init_state's checks
      st = run_cta(g, max_iters, tol, p, &di, &ms);
      if (st != GN_OK) return st;
    }
    kused = GN_KERNEL_CTA;
  } else if (max_iters > start_iter && g->n > 0) {
    st = run_iterations(g, start_iter, max_iters, tol, p, parity0, &di, &ms, &kused);
    if (st != GN_OK) return st;
    if (!(di.status & DEV_TIMEOUT)) g->state_parity = parity0 ^ di.final_parity;
  } else {
    GN_CUDA(cudaMemcpyAsync(&di, g->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
    if (di.status == 0 && g->n > 0) {
      st = state_stats(g, g->d_x, p.theta_bin, &di.objective, &di.nonbin);
      if (st != GN_OK) return st;
      di.binary = di.nonbin == 0;
    }
  }
  if (di.status & DEV_NOT_NORMALIZABLE)
    return fail(GN_ERR_NOT_NORMALIZABLE, "gn_run: x0 is negative, not finite or not normalizable");
  if (di.status & DEV_TIMEOUT)
    return fail(GN_ERR_TIMEOUT, "gn_run: a grid-barrier wait hit its limit; the run was abandoned");
  g->has_state = true;
  g->state_cta = kused == GN_KERNEL_CTA;

  gn_status result;
  if (di.iters == 0) {
    di.converged = 0;
    result = GN_WARN_NOT_CONVERGED;
  } else if (!di.converged) {
    result = GN_WARN_NOT_CONVERGED;
  } else {
    const double gl = host_gamma(p, start_iter + di.iters - 1);
    result = (di.nonbin == 0 && gl * (1.0 - p.theta_bin) > p.theta_bin) ? GN_OK : GN_WARN_NOT_BINARY;
  }

  if (x_out && g->n > 0) {
    float* tmp = g->io_mem == GN_DEVICE ? x_out : g->d_io;
    k_to_caller<<<(g->n + 255) / 256, 256, 0, g->stream>>>(g->n, g->d_x, g->d_iperm, tmp);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
    if (g->io_mem == GN_HOST) {
      GN_CUDA(cudaMemcpyAsync(x_out, tmp, sizeof(float) * g->n, cudaMemcpyDeviceToHost, g->stream));
    }
    GN_CUDA(cudaStreamSynchronize(g->stream));
  }
  if (info) {
    memset(info, 0, sizeof *info);
    info->iters = di.iters;
    info->converged = di.converged;
    info->binary = di.binary;
    info->status = result;
    info->resid_inf = di.resid_inf;
    info->resid_l1 = di.resid_l1;
    info->objective = di.objective;
    info->energy = di.energy;
    info->safe_div_hits = (long long)di.hits;
    info->device_ms = ms;
    info->kernel = kused;
  }
  return result;
}

// ==========================================================================================
// gn_run_noalloc: the persistent iteration without any device allocation.
//
// Who needs this: code that is handed device buffers by a host runtime and may not allocate
// device memory itself -- for instance a plugin or custom operator living inside another
// framework's memory pool, a real-time service that allocates everything at start-up, or a
// caller that issues work while the process's allocator is locked.  gn_create allocates the
// handle's buffers with cudaMalloc; this entry point instead carves every scratch buffer the
// persistent kernel needs (weighted states, v as a float pair, per-CTA check partials, the
// grid-barrier counter, the run summary) out of one fixed array in the library's device
// globals, which every GPU that loads the library holds until the process exits.
//
// Consequences a caller must respect:
//   - at most kNoAllocMaxN vertices (larger graphs are rejected with GN_ERR_TOO_LARGE);
//   - every call on a device shares the same array and leaves its contents behind, so calls
//     whose device work overlaps (two host threads, or two streams) race and corrupt each
//     other: serialise them;
//   - the first call on each device resolves the array's device address with
//     cudaGetSymbolAddress (and sets the kernel's shared-memory attribute);
//   - every call reads row_ptr[n] and the run summary back to the host and synchronises the
//     stream, so no call may be made while the stream is being captured.
namespace gn {

static constexpr int kNoAllocMaxN = 65536;
static constexpr int kNoAllocMaxCTAs = 256;
static constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }
static constexpr size_t kNaVec = align256(sizeof(float) * kNoAllocMaxN);
static constexpr size_t kNaOffY0 = 0;
static constexpr size_t kNaOffY1 = kNaOffY0 + kNaVec;
static constexpr size_t kNaOffYlo = kNaOffY1 + kNaVec;
static constexpr size_t kNaOffYexp = kNaOffYlo + kNaVec;
static constexpr size_t kNaOffX = kNaOffYexp + kNaVec;
static constexpr size_t kNaOffV = kNaOffX + kNaVec;
static constexpr size_t kNaOffVlo = kNaOffV + kNaVec;
static constexpr size_t kNaOffPartials = kNaOffVlo + kNaVec;
static constexpr size_t kNaOffPart = kNaOffPartials + align256(sizeof(CheckPartial) * 2 * kNoAllocMaxCTAs);
static constexpr size_t kNaOffInfo = kNaOffPart + align256(sizeof(int32_t) * (kNoAllocMaxCTAs + 1));
static constexpr int kNoAllocMaxGamma = 16384;
static constexpr size_t kNaOffBar = kNaOffInfo + align256(sizeof(DevInfo));
static constexpr size_t kNaOffGtab = kNaOffBar + 256;
static constexpr size_t kNoAllocScratchBytes = kNaOffGtab + align256(sizeof(float2) * kNoAllocMaxGamma);

// the fixed scratch (about 2 MB per device)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// range, order and self-loop check of the caller's CSR (flags go to the run summary's status).
// nnz = row_ptr[n] as read on the host: a row whose range leaves [0, nnz) is malformed and its
// entries are not read, so a row_ptr that decreases further on cannot send a row past col_idx.
__global__ void k_na_check_rows(int n, int nnz, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int b = rp[i], e = rp[i + 1];
  if (b < 0 || e < b || e > nnz || (i == 0 && b != 0)) {
    atomicOr(status, DEV_BAD_CSR);
    return;
  }
  int prev = -1;
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j < 0 || j >= n) {
      atomicOr(status, DEV_BAD_CSR);
      return;
    }
    if (j == i || j <= prev) atomicOr(status, DEV_NOT_SIMPLE);
    prev = j;
  }
}

// symmetry, only after the range check passed (the kernel reads the flag first)
__global__ void k_na_check_symmetry(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                    int* status) {
  if (dev::ld_relaxed_int(status) & DEV_BAD_CSR) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = rp[i]; k < rp[i + 1]; ++k) {
    int j = ci[k];
    int a = rp[j], b = rp[j + 1] - 1;
    bool found = false;
    while (a <= b) {
      int m = (a + b) >> 1;
      int c = ci[m];
      if (c == i) { found = true; break; }
      if (c < i) a = m + 1; else b = m - 1;
    }
    if (!found) {
      atomicOr(status, DEV_NOT_SIMPLE);
      return;
    }
  }
}

// v = sqrt(w) as a float pair, start state (x0 or 1/(deg+1), Def. 1 check), equal-rows
// partition; skipped when the CSR is malformed
__global__ void k_na_init(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                          const float* __restrict__ w, const float* __restrict__ x0, float* __restrict__ v,
                          float* __restrict__ vlo, float* __restrict__ x, float* __restrict__ y,
                          float* __restrict__ ylo, float* __restrict__ yexp, int32_t* __restrict__ part,
                          int nblocks, int rows_per, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the partition is written first and unconditionally: the iteration kernel reads it
  // (and returns at once when the status word is set)
  if (i <= nblocks) part[i] = min(i * rows_per, n);
  if (dev::ld_relaxed_int(status) & DEV_BAD_CSR) return;
  if (i >= n) return;
  float wi = w[i];
  dev::f2 vv = {1.0f, 0.0f};
  if (!(wi > 0.0f) || !isfinite(wi)) atomicOr(status, DEV_BAD_WEIGHT);
  else vv = dev::split_f64(sqrt((double)wi));
  v[i] = vv.hi;
  vlo[i] = vv.lo;
  const int b = rp[i], e = rp[i + 1];
  float xi = x0 ? x0[i] : __frcp_rn((float)(e - b + 1));
  bool bad = !(xi >= 0.0f) || !isfinite(xi);
  if (x0 && !bad && !(xi > 0.0f)) {
    bool pos = false;
    for (int k = b; k < e && !pos; ++k) pos = x0[ci[k]] > 0.0f;
    bad = !pos;
  }
  if (bad) atomicOr(status, DEV_NOT_NORMALIZABLE);
  x[i] = xi;
  dev::f2 yy = dev::mul_f2(vv, dev::f2{xi, 0.0f});
  y[i] = yy.hi;
  ylo[i] = yy.lo;
  yexp[i] = 0.0f;
}

// the result, clamped to [0, 1], into the caller's buffer; nothing is written when the run
// failed (the status word is set)
__global__ void k_na_out(int n, const float* __restrict__ x, float* __restrict__ out, const int* status) {
  if (dev::ld_relaxed_int(status) != 0) return;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = fminf(fmaxf(x[i], 0.0f), 1.0f);
}

static std::mutex g_na_mutex;
static unsigned char* g_na_ptr[64] = {nullptr};
static int g_na_sms[64] = {0};

}  // namespace gn

extern "C" gn_status gn_run_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                    const float* w, const float* x0, int max_iters, double tol,
                                    const gn_params* pin, int start_iter, float* x_out,
                                    gn_run_info* info, void* stream_v) {
  using namespace gn;
  if (n < 0 || (n > 0 && (!row_ptr || !w || !x_out)))
    return fail(GN_ERR_ARG, "gn_run_noalloc: bad argument");
  if (n > kNoAllocMaxN)
    return fail(GN_ERR_TOO_LARGE, "gn_run_noalloc: n exceeds the fixed scratch (65536 vertices); "
                                  "use gn_create / gn_run");
  gn_params p;
  if (pin) p = *pin; else gn_default_params(&p);
  if (start_iter < 0 || max_iters < start_iter || p.check_every < 1 || !(p.theta_bin < 0.5) || p.resume ||
      !std::isfinite(p.gamma0) || !std::isfinite(p.gamma1) || p.gamma1 < 0 || p.gamma0 < 0 ||
      (p.gamma_mode != GN_GAMMA_PURSUIT && p.gamma_mode != GN_GAMMA_FIXED))
    return fail(GN_ERR_ARG, "gn_run_noalloc: bad argument (resume is not available without a handle)");
  cudaStream_t stream = (cudaStream_t)stream_v;
  int dev_id = 0;
  GN_CUDA(cudaGetDevice(&dev_id));
  if (dev_id < 0 || dev_id >= 64) return fail(GN_ERR_ARG, "gn_run_noalloc: device index out of range");

  // one-time set-up per device: the scratch's device address and the kernel attribute
  unsigned char* base = nullptr;
  int sms = 0;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev_id]) {
      void* ptr = nullptr;
      GN_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
      GN_CUDA(cudaDeviceGetAttribute(&g_na_sms[dev_id], cudaDevAttrMultiProcessorCount, dev_id));
      for (int G = 1; G <= 32; G <<= 1)
        GN_CUDA(cudaFuncSetAttribute((const void*)pick_kernel(G, MODE_GMEM),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLimit));
      g_na_ptr[dev_id] = static_cast<unsigned char*>(ptr);
    }
    base = g_na_ptr[dev_id];
    sms = g_na_sms[dev_id];
  }
  float* s_y0 = reinterpret_cast<float*>(base + kNaOffY0);
  float* s_y1 = reinterpret_cast<float*>(base + kNaOffY1);
  float* s_ylo = reinterpret_cast<float*>(base + kNaOffYlo);
  float* s_yexp = reinterpret_cast<float*>(base + kNaOffYexp);
  float* s_x = reinterpret_cast<float*>(base + kNaOffX);
  float* s_v = reinterpret_cast<float*>(base + kNaOffV);
  float* s_vlo = reinterpret_cast<float*>(base + kNaOffVlo);
  CheckPartial* s_partials = reinterpret_cast<CheckPartial*>(base + kNaOffPartials);
  int32_t* s_part = reinterpret_cast<int32_t*>(base + kNaOffPart);
  DevInfo* s_info = reinterpret_cast<DevInfo*>(base + kNaOffInfo);
  unsigned* s_bar = reinterpret_cast<unsigned*>(base + kNaOffBar);
  float2* s_gtab = reinterpret_cast<float2*>(base + kNaOffGtab);

  if (n == 0) {
    if (info) {
      memset(info, 0, sizeof *info);
      info->status = GN_WARN_NOT_CONVERGED;
    }
    return GN_WARN_NOT_CONVERGED;
  }
  int32_t nnz = 0;
  GN_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, stream));
  GN_CUDA(cudaStreamSynchronize(stream));
  if (nnz < 0 || (nnz > 0 && !col_idx)) return fail(GN_ERR_ARG, "gn_run_noalloc: bad row_ptr or col_idx");

  // launch shape: equal row ranges, CSR read from global memory
  const int nb = std::max(1, std::min({sms, kNoAllocMaxCTAs, (n + 63) / 64}));
  const int rows_per = (n + nb - 1) / nb;
  const double avg = (double)nnz / n;
  int G = 1;
  while (G < 32 && G * 3 < avg) G <<= 1;
  const int R = (rows_per + 3) & ~3;
  const size_t smem = sizeof(float) * 6 * (size_t)R + sizeof(int) * ((size_t)R + 4) + sizeof(int) * (size_t)R;
  KernelFn fn = pick_kernel(G, MODE_GMEM);
  int per_sm = 0;
  GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
  if (per_sm < 1 || nb > per_sm * sms) return fail(GN_ERR_TOO_LARGE, "gn_run_noalloc: kernel does not fit");
  if ((int64_t)(max_iters - start_iter) * nb >= (int64_t)1 << 31)
    return fail(GN_ERR_TOO_LARGE, "gn_run_noalloc: too many iterations for one call");
  const int glen = (p.gamma_mode == GN_GAMMA_FIXED || p.ramp_iters <= 1)
                       ? 1
                       : std::max(1, std::min(max_iters, p.ramp_iters));
  if (glen > kNoAllocMaxGamma)
    return fail(GN_ERR_TOO_LARGE, "gn_run_noalloc: the gamma ramp needs more than 16384 table entries");

  // what must start at zero: the run summary (status, counters) and the barrier counter
  GN_CUDA(cudaMemsetAsync(s_info, 0, sizeof(DevInfo), stream));
  GN_CUDA(cudaMemsetAsync(s_bar, 0, sizeof(unsigned) * 8, stream));  // counter and check words
  const unsigned grid = (unsigned)std::max(n, nb + 1);
  k_na_check_rows<<<(n + 255) / 256, 256, 0, stream>>>(n, nnz, row_ptr, col_idx, &s_info->status);
  GN_LAUNCHED();
  k_na_check_symmetry<<<(n + 255) / 256, 256, 0, stream>>>(n, row_ptr, col_idx, &s_info->status);
  GN_LAUNCHED();
  k_na_init<<<(grid + 255) / 256, 256, 0, stream>>>(n, row_ptr, col_idx, w, x0, s_v, s_vlo, s_x, s_y0,
                                                     s_ylo, s_yexp, s_part, nb, rows_per, &s_info->status);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());

  DevInfo di;
  memset(&di, 0, sizeof di);
  float ms = 0.0f;
  if (max_iters > start_iter) {
    IterParams P;
    P.row_ptr = row_ptr;
    P.col_idx = col_idx;
    P.v = s_v;
    P.vlo = s_vlo;
    P.w = w;
    P.part = s_part;
    P.y0 = s_y0;
    P.y1 = s_y1;
    P.x = s_x;
    P.ylo = s_ylo;
    P.yexp = s_yexp;
    P.hoff = nullptr;
    P.hblob = nullptr;
    P.halo_pad = 0;
    P.iterflag = nullptr;
    P.inbox = nullptr;
    P.inbox_len = 0;
    k_gamma_table<<<(glen + 255) / 256, 256, 0, stream>>>(glen, p.gamma_mode, p.gamma0, p.gamma1,
                                                          p.ramp_iters, s_gtab);
    GN_LAUNCHED();
    P.gtab = s_gtab;
    P.gtab_len = glen;
    P.partials = s_partials;
    P.bar = s_bar;
    P.status = &s_info->status;
    P.info = s_info;
    P.n = n;
    P.nblocks = nb;
    P.k_start = start_iter;
    P.k_end = max_iters;
    P.gamma_mode = p.gamma_mode;
    P.gamma0 = p.gamma0;
    P.gamma1 = p.gamma1;
    P.ramp = p.ramp_iters;
    P.check_every = p.check_every;
    set_stop_thresholds(P, p.theta_bin, tol);
    P.heavy = 16 * G;
    P.rows_pad = R;
    P.spin_limit = p.spin_limit > 0 ? p.spin_limit : (1ll << 22);
    P.unreachable = p.debug_unreachable_barrier ? 1 : 0;
    P.bad_tag = 0;
    void* args[] = {(void*)&P};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = info != nullptr;
    if (timed) {
      GN_CUDA(cudaEventCreate(&e0));
      GN_CUDA(cudaEventCreate(&e1));
      GN_CUDA(cudaEventRecord(e0, stream));
    }
    GN_CUDA(cudaLaunchCooperativeKernel((const void*)fn, dim3(nb), dim3(kThreads), args, smem, stream));
    GN_LAUNCHED();
    if (timed) GN_CUDA(cudaEventRecord(e1, stream));
    k_na_out<<<(n + 255) / 256, 256, 0, stream>>>(n, s_x, x_out, &s_info->status);
    GN_LAUNCHED();
    GN_CUDA(cudaMemcpyAsync(&di, s_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, stream));
    GN_CUDA(cudaStreamSynchronize(stream));
    if (timed) {
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
  } else {
    k_na_out<<<(n + 255) / 256, 256, 0, stream>>>(n, s_x, x_out, &s_info->status);  // the start state
    GN_LAUNCHED();
    GN_CUDA(cudaMemcpyAsync(&di, s_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, stream));
    GN_CUDA(cudaStreamSynchronize(stream));
  }
  if (di.status & DEV_BAD_CSR) return fail(GN_ERR_ARG, "gn_run_noalloc: malformed CSR");
  if (di.status & DEV_NOT_SIMPLE) return fail(GN_ERR_NOT_SIMPLE, "gn_run_noalloc: graph is not simple");
  if (di.status & DEV_BAD_WEIGHT) return fail(GN_ERR_WEIGHT, "gn_run_noalloc: weight <= 0 or not finite");
  if (di.status & DEV_NOT_NORMALIZABLE)
    return fail(GN_ERR_NOT_NORMALIZABLE, "gn_run_noalloc: x0 is negative, not finite or not normalizable");
  if (di.status & DEV_TIMEOUT) return fail(GN_ERR_TIMEOUT, "gn_run_noalloc: a grid-barrier wait hit its limit");
  gn_status result;
  if (di.iters == 0 || !di.converged) {
    result = GN_WARN_NOT_CONVERGED;
  } else {
    const double gl = host_gamma(p, start_iter + di.iters - 1);
    result = (di.nonbin == 0 && gl * (1.0 - p.theta_bin) > p.theta_bin) ? GN_OK : GN_WARN_NOT_BINARY;
  }
  if (info) {
    memset(info, 0, sizeof *info);
    info->iters = di.iters;
    info->converged = di.converged;
    info->binary = di.binary;
    info->status = result;
    info->resid_inf = di.resid_inf;
    info->resid_l1 = di.resid_l1;
    info->objective = di.objective;
    info->energy = di.energy;
    info->safe_div_hits = (long long)di.hits;
    info->device_ms = ms;
    info->kernel = GN_KERNEL_PERSISTENT;
  }
  return result;
}
