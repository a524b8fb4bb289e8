// gn_adjoint.cu -- differentiable GN: the recorded forward (gn_run with params.record = 1) and
// its reverse mode (gn_backward).
//
// Forward, weighted state (App. B): y_{t+1} = v (.) y_t / d_t with d_t = (I + gamma_t A) y_t;
// the run stores the state every S = ceil(sqrt(T)) steps (sqrt(T) checkpointing).
// Reverse, derived from the step's Jacobian (App. G, Lemma 2 in its general form) and carried
// in log space: with u = log y the step is u'_i = log v_i + u_i - log d_i, so
//   du'_i/du_i = 1 - x'_i = gamma s_i / d_i,   du'_i/du_j = -gamma y_j / d_i  (j in N(i)),
//   du'_i/dv_i = 1 / v_i,
// every coefficient lies in [-1, 1] (d_i >= gamma y_j), so the adjoint h = dL/du = gbar_y (.) y
// cannot overflow however small the states get (the y-space adjoint multiplies by 1/d_i):
//   h_j = h'_j gamma s_j / d_j - gamma y_j sum_{i in N(j)} h'_i / d_i,   gbar_v += h' / v.
// A safe-division row (d_i <= 1e-9, y'_i = v_i / 2) passes nothing to u and h'_i / v_i to v.
// The ends: h_T = dL/dx_T (.) x_T and gbar_v = -dL/dx_T (.) x_T / v (x_T = y_T / v);
// dL/dx_0 = h_0 / x_0, gbar_v += h_0 / v (y_0 = v x_0); dL/dw = gbar_v / (2 v).
// Each backward segment is recomputed from its checkpoint; every step is two gathers.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gn_internal.cuh"
#include "gn_iter_common.cuh"

namespace gn {

struct RecordState {
  int n = 0;
  int k_start = 0, T = 0, S = 0, ncp = 0;
  gn_params p;
  float* cp_hi = nullptr;   // [ncp][n] states after c*S steps (c = 0: y_0)
  float* cp_lo = nullptr;
  float* seg_hi = nullptr;  // [S + 1][n] states of the segment being reversed
  float* seg_lo = nullptr;
  float* x0 = nullptr;      // start x_0 (internal order)
  float* xT = nullptr;      // x_T
  float* g = nullptr;       // log-space adjoint h = dL/du of the current state (u = log y)
  float* a = nullptr;
  float* t = nullptr;
  float* gv = nullptr;      // accumulated adjoint of v
  float2* gtab = nullptr;   // gamma_k table for k_start .. k_start + T - 1
  bool valid = false;
};

static constexpr int kAdjThreads = 256;

// The recorded forward keeps its states as plain float pairs in FP32's range (the log-space
// adjoint below reads y = hi + lo); a vertex below FP32's smallest normal contributes nothing to
// the gradient.  Otherwise the arithmetic of gn_run's update: d = y + gamma s, x' = y / d,
// y' = v x', the safe division at d <= 1e-9.
__device__ __forceinline__ void step_pair(dev::f2& y, const dev::f2 v, float& x, float sn, dev::f2 gam,
                                          unsigned long long& hits) {
  dev::f2 p = dev::two_prod(gam.hi, sn);
  p.lo = dev::ffma(gam.lo, sn, p.lo);
  dev::f2 d = dev::two_sum(y.hi, p.hi);
  d = dev::fast_two_sum(d.hi, dev::fadd(d.lo, dev::fadd(y.lo, p.lo)));
  const bool ok = d.hi > kSafeDiv;
  const dev::f2 q = dev::div_f2(y, ok ? d : dev::f2{1.0f, 0.0f});
  const dev::f2 xn = ok ? q : dev::f2{0.5f, 0.0f};
  hits += ok ? 0ull : 1ull;
  y = dev::mul_f2(v, xn);
  x = xn.hi;
}

// one forward step, thread per row: y_out = v y_in / ((I + gamma A) y_in) (float pairs)
__global__ void k_step(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const float* __restrict__ vh, const float* __restrict__ vl, float2 gam,
                       const float* __restrict__ yh, const float* __restrict__ yl, float* __restrict__ oh,
                       float* __restrict__ ol, float* __restrict__ x_out, unsigned long long* hits) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int e = rp[i]; e < rp[i + 1]; ++e) s += yh[ci[e]];
  dev::f2 y = {yh[i], yl[i]};
  float x = 0.0f;
  unsigned long long h = 0;
  step_pair(y, dev::f2{vh[i], vl[i]}, x, s, dev::f2{gam.x, gam.y}, h);
  oh[i] = y.hi;
  ol[i] = y.lo;
  if (x_out) x_out[i] = x;
  if (h && hits) atomicAdd(hits, h);
}

// adjoint part 1 at step t: recompute s and d from y_t, then r = h' / d and the own term
// o = h' gamma s / d, and the v-adjoint
__global__ void k_adj1(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                       const float* __restrict__ vh, float2 gam, const float* __restrict__ yh,
                       const float* __restrict__ yl, const float* __restrict__ h, float* __restrict__ r,
                       float* __restrict__ o, float* __restrict__ gv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float s = 0.0f;
  for (int e = rp[i]; e < rp[i + 1]; ++e) s += yh[ci[e]];
  const float y = yh[i] + yl[i];
  const float gs = fmaf(gam.y, s, gam.x * s);  // gamma s
  const float d = y + gs;
  const float hi = h[i];
  if (d > kSafeDiv) {
    const float inv = 1.0f / d;
    r[i] = hi * inv;
    o[i] = hi * (gs * inv);
  } else {
    r[i] = 0.0f;
    o[i] = 0.0f;
  }
  gv[i] += hi / vh[i];
}

// adjoint part 2: h_j = o_j - gamma y_j sum_{i in N(j)} r_i
__global__ void k_adj2(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci, float2 gam,
                       const float* __restrict__ yh, const float* __restrict__ yl, const float* __restrict__ r,
                       const float* __restrict__ o, float* __restrict__ h) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float q = 0.0f;
  for (int e = rp[i]; e < rp[i + 1]; ++e) q += r[ci[e]];
  const float y = yh[i] + yl[i];
  h[i] = o[i] - fmaf(gam.y, q, gam.x * q) * y;
}

// the output end: h_T = dL/dx_T x_T, gbar_v = -dL/dx_T x_T / v
__global__ void k_adj_out(int n, const float* __restrict__ gx_int, const float* __restrict__ vh,
                          const float* __restrict__ xT, float* __restrict__ h, float* __restrict__ gv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float hx = gx_int[i] * xT[i];
  h[i] = hx;
  gv[i] = -hx / vh[i];
}

// the input end (y_0 = v x_0): dL/dx_0 = h_0 / x_0, gbar_v += h_0 / v, dL/dw = gbar_v / (2 v);
// outputs in caller order
__global__ void k_adj_in(int n, const float* __restrict__ h, const float* __restrict__ vh,
                         const float* __restrict__ x0, const float* __restrict__ gv,
                         const int32_t* __restrict__ iperm, float* __restrict__ dw, float* __restrict__ dx0) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const int i = iperm ? iperm[c] : c;
  const float h0 = h[i];
  if (dx0) dx0[c] = x0[i] > 0.0f ? h0 / x0[i] : 0.0f;
  if (dw) dw[c] = (gv[i] + h0 / vh[i]) / (2.0f * vh[i]);
}

__global__ void k_gather_perm(int n, const float* __restrict__ src, const int32_t* __restrict__ perm,
                              float* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[perm ? perm[i] : i];
}

__global__ void k_record_gamma(int T, int k0, int mode, double g0, double g1, int ramp, float2* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= T) return;
  const dev::f2 p = dev::split_f64(dev::gamma_at(mode, g0, g1, ramp, k0 + j));
  out[j] = make_float2(p.hi, p.lo);
}

static void free_record(RecordState* r) {
  if (!r) return;
  void* d[] = {r->cp_hi, r->cp_lo, r->seg_hi, r->seg_lo, r->x0, r->xT, r->g, r->a, r->t, r->gv, r->gtab};
  for (void* p : d)
    if (p) cudaFree(p);
  delete r;
}

static unsigned blocks(int n) { return (unsigned)std::max(1, (n + kAdjThreads - 1) / kAdjThreads); }

// The recorded forward: T = k_end - k_start steps from the state init_state left in d_x / d_y[0] /
// d_ylo, checkpoints every S steps.  Leaves x_T in d_x and the final state as gn_run does.
gn_status record_forward(gn_graph* g, int k_start, int k_end, const gn_params& p, DevInfo* out, float* ms) {
  const int n = g->n;
  const int T = k_end - k_start;
  RecordState* r = g->rec;
  if (!r || r->n != n || r->T != T) {
    free_record(r);
    g->rec = nullptr;
    r = new RecordState();
    g->rec = r;
    r->n = n;
    r->T = T;
    r->S = std::max(1, (int)std::ceil(std::sqrt((double)T)));
    r->ncp = T / r->S + 1;
    const size_t nb = sizeof(float) * (size_t)std::max(n, 1);
    GN_CUDA(cudaMalloc(&r->cp_hi, nb * r->ncp));
    GN_CUDA(cudaMalloc(&r->cp_lo, nb * r->ncp));
    GN_CUDA(cudaMalloc(&r->seg_hi, nb * (r->S + 1)));
    GN_CUDA(cudaMalloc(&r->seg_lo, nb * (r->S + 1)));
    GN_CUDA(cudaMalloc(&r->x0, nb));
    GN_CUDA(cudaMalloc(&r->xT, nb));
    GN_CUDA(cudaMalloc(&r->g, nb));
    GN_CUDA(cudaMalloc(&r->a, nb));
    GN_CUDA(cudaMalloc(&r->t, nb));
    GN_CUDA(cudaMalloc(&r->gv, nb));
    GN_CUDA(cudaMalloc(&r->gtab, sizeof(float2) * std::max(T, 1)));
  }
  r->valid = false;
  r->k_start = k_start;
  r->p = p;
  k_record_gamma<<<blocks(T), kAdjThreads, 0, g->stream>>>(T, k_start, p.gamma_mode, p.gamma0, p.gamma1,
                                                           p.ramp_iters, r->gtab);
  GN_LAUNCHED();
  std::vector<float2> gam(std::max(T, 1));
  GN_CUDA(cudaMemcpyAsync(gam.data(), r->gtab, sizeof(float2) * T, cudaMemcpyDeviceToHost, g->stream));
  const size_t nb = sizeof(float) * (size_t)n;
  GN_CUDA(cudaMemcpyAsync(r->x0, g->d_x, nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(r->cp_hi, g->d_y[0], nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(r->cp_lo, g->d_ylo, nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemsetAsync(&g->d_info->hits, 0, sizeof(unsigned long long), g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  GN_CUDA(cudaEventRecord(g->ev0, g->stream));
  // states ping-pong in the segment buffer's first two slots
  float *ah = r->seg_hi, *al = r->seg_lo, *bh = r->seg_hi + n, *bl = r->seg_lo + n;
  GN_CUDA(cudaMemcpyAsync(ah, g->d_y[0], nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(al, g->d_ylo, nb, cudaMemcpyDeviceToDevice, g->stream));
  for (int j = 0; j < T; ++j) {
    k_step<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, g->d_v, g->d_vlo, gam[j], ah, al,
                                                     bh, bl, j == T - 1 ? g->d_x : nullptr, &g->d_info->hits);
    GN_LAUNCHED();
    std::swap(ah, bh);
    std::swap(al, bl);
    if ((j + 1) % r->S == 0) {
      const int c = (j + 1) / r->S;
      GN_CUDA(cudaMemcpyAsync(r->cp_hi + (size_t)c * n, ah, nb, cudaMemcpyDeviceToDevice, g->stream));
      GN_CUDA(cudaMemcpyAsync(r->cp_lo + (size_t)c * n, al, nb, cudaMemcpyDeviceToDevice, g->stream));
    }
  }
  GN_CUDA(cudaEventRecord(g->ev1, g->stream));
  GN_CUDA(cudaGetLastError());
  // final state where gn_run leaves it
  GN_CUDA(cudaMemcpyAsync(g->d_y[0], ah, nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(g->d_ylo, al, nb, cudaMemcpyDeviceToDevice, g->stream));
  GN_CUDA(cudaMemsetAsync(g->d_yexp, 0, nb, g->stream));  // plain float pairs: no scaled rows
  GN_CUDA(cudaMemcpyAsync(r->xT, g->d_x, nb, cudaMemcpyDeviceToDevice, g->stream));
  g->state_parity = 0;
  GN_CUDA(cudaMemcpyAsync(out, g->d_info, sizeof(DevInfo), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (ms) GN_CUDA(cudaEventElapsedTime(ms, g->ev0, g->ev1));
  out->iters = T;
  out->converged = 0;
  out->final_parity = 0;
  r->valid = true;
  return GN_OK;
}

}  // namespace gn

void gn_free_record(gn_graph* g) {
  if (g && g->rec) {
    gn::free_record(g->rec);
    g->rec = nullptr;
  }
}

extern "C" gn_status gn_backward(gn_graph* g, const float* dL_dxT, float* dL_dw, float* dL_dx0) {
  using namespace gn;
  if (!g) return fail(GN_ERR_ARG, "gn_backward: NULL handle");
  if (!g->rec || !g->rec->valid) return fail(GN_ERR_NO_RECORD, "gn_backward: no recorded forward run");
  if (!dL_dxT) return fail(GN_ERR_ARG, "gn_backward: dL_dxT is NULL");
  GN_CUDA(cudaSetDevice(g->device));
  RecordState* r = g->rec;
  const int n = g->n, T = r->T, S = r->S;
  if (n == 0) return GN_OK;
  const size_t nb = sizeof(float) * (size_t)n;
  std::vector<float2> gam(std::max(T, 1));
  GN_CUDA(cudaMemcpyAsync(gam.data(), r->gtab, sizeof(float2) * T, cudaMemcpyDeviceToHost, g->stream));
  // dL/dx_T into internal order
  const float* gx_dev = nullptr;
  gn_status st = upload_or_alias(g, dL_dxT, nb, (const void**)&gx_dev);
  if (st != GN_OK) return st;
  k_gather_perm<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, gx_dev, g->d_perm, r->a);
  GN_LAUNCHED();
  k_adj_out<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, r->a, g->d_v, r->xT, r->g, r->gv);
  GN_LAUNCHED();
  GN_CUDA(cudaStreamSynchronize(g->stream));
  // segments from the last to the first
  const int nseg = (T + S - 1) / S;
  for (int sgi = nseg - 1; sgi >= 0; --sgi) {
    const int j0 = sgi * S, j1 = std::min(T, j0 + S);
    // recompute states j0 .. j1-1 of the segment from checkpoint sgi
    GN_CUDA(cudaMemcpyAsync(r->seg_hi, r->cp_hi + (size_t)sgi * n, nb, cudaMemcpyDeviceToDevice, g->stream));
    GN_CUDA(cudaMemcpyAsync(r->seg_lo, r->cp_lo + (size_t)sgi * n, nb, cudaMemcpyDeviceToDevice, g->stream));
    for (int j = j0; j < j1 - 1; ++j) {
      const int q = j - j0;
      k_step<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, g->d_v, g->d_vlo, gam[j],
                                                       r->seg_hi + (size_t)q * n, r->seg_lo + (size_t)q * n,
                                                       r->seg_hi + (size_t)(q + 1) * n,
                                                       r->seg_lo + (size_t)(q + 1) * n, nullptr, nullptr);
      GN_LAUNCHED();
    }
    // reverse through the segment
    for (int j = j1 - 1; j >= j0; --j) {
      const int q = j - j0;
      k_adj1<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, g->d_v, gam[j],
                                                       r->seg_hi + (size_t)q * n, r->seg_lo + (size_t)q * n, r->g,
                                                       r->a, r->t, r->gv);
      GN_LAUNCHED();
      k_adj2<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, gam[j],
                                                       r->seg_hi + (size_t)q * n, r->seg_lo + (size_t)q * n, r->a,
                                                       r->t, r->g);
      GN_LAUNCHED();
    }
  }
  GN_CUDA(cudaGetLastError());
  // outputs in caller order
  float* dw = dL_dw;
  float* dx = dL_dx0;
  float* tmp_w = nullptr;
  float* tmp_x = nullptr;
  if (g->io_mem == GN_HOST) {
    tmp_w = dL_dw ? r->a : nullptr;
    tmp_x = dL_dx0 ? r->t : nullptr;
    dw = tmp_w;
    dx = tmp_x;
  }
  k_adj_in<<<blocks(n), kAdjThreads, 0, g->stream>>>(n, r->g, g->d_v, r->x0, r->gv, g->d_iperm, dw, dx);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  if (g->io_mem == GN_HOST) {
    if (dL_dw) GN_CUDA(cudaMemcpyAsync(dL_dw, tmp_w, nb, cudaMemcpyDeviceToHost, g->stream));
    if (dL_dx0) GN_CUDA(cudaMemcpyAsync(dL_dx0, tmp_x, nb, cudaMemcpyDeviceToHost, g->stream));
  }
  GN_CUDA(cudaStreamSynchronize(g->stream));
  return GN_OK;
}
