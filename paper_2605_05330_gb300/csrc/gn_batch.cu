// gn_batch.cu -- batched Graph Normalization: thousands of independent instances of uneven
// size in one persistent launch.
//
// A CTA takes an instance from an atomic work queue (instances ordered by decreasing work,
// longest-processing-time first), keeps the whole instance in shared memory and iterates it to
// its own stop test (per-instance convergence: a finished instance frees its CTA for the next
// one), then writes its state and summary.  No grid-wide synchronisation exists.
// Packing: instances up to a size threshold form a second queue, run a warp per instance (a
// CTA's warps take them one by one, each in its own slice of the CTA's shared memory, with warp
// synchronisation only) once the CTA queue is empty.  A warp sums a row with the same lanes and
// in the same order as a CTA, so both modes give the same iterates bit for bit.  The CTA size
// and the threshold are the autotuner's choices (gn_batch_tune).
//
// Two instance kinds:
//   GN_INSTANCE_CSR         a general graph given as CSR (local ids); G lanes per row
//   GN_INSTANCE_ASSIGNMENT  the assignment conflict graph of a k x k matrix (Sec. 2: the line
//                           graph of K_{k,k}; cells adjacent when they share a row or column).
//                           The neighbour sum of cell (r, c) is R_r + C_c - 2 y_rc with R and C
//                           the row and column sums (the cross-normalisation of Sec. 2), so the
//                           instance needs no edge list and O(k^2) work per iteration.
// The update, schedule and stop test are those of gn_run (float-pair own state, FP32 gathers).
// The run sequence is captured once into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "gn_internal.cuh"
#include "gn_iter_common.cuh"

namespace gn {

struct BatchInfoDev {
  int iters;
  int converged;
  int binary;
  unsigned nonbin;
  unsigned long long hits;
  float resid_inf;
  float pad;
  double objective;
  double resid_l1;   // sum |x' - x| of the last check
  double energy;     // E~ of the state entering the last check's step
};

struct BatchParams {
  int count;
  const int64_t* vtx_off;   // [count + 1]
  const int64_t* ent_off;   // [count + 1]
  const int32_t* row_ptr;   // per instance i: n_i + 1 local offsets at vtx_off[i] + i
  const int32_t* col_idx;   // per instance i: local ids at ent_off[i]
  const int32_t* kind;
  const int32_t* order;     // processing order
  const int32_t* group;     // lanes per light row, per instance
  const float* w;
  const float* v;
  const float* vlo;
  float* x;                 // in: x0, out: final x (concatenated)
  BatchInfoDev* info;
  unsigned* queue;
  const float2* gtab;
  int gtab_len;
  int k_end;
  int check_every;
  double theta;
  double tol;
  float thr_hi, thr_lo;     // gamma (1 - theta) > theta <=> gamma > thr (float pair), no FP64
  float tol_f;              // r <= tol <=> r <= tol_f for an FP32 r
  int res_test;             // tol >= 0
  int nmax;                 // largest instance (the state arrays of the shared-memory layout)
  int ncsr;                 // largest CSR instance (its neighbour sums and row offsets)
  int idcap;                // local ids held in shared memory up to this many entries
  int nbig;                 // order[0, nbig): CTA per instance; order[nbig, count): warp per instance
  int wbytes;               // shared memory of one warp in warp mode (multiple of 16)
};

static constexpr int kBatchMaxThreads = 1024;

__device__ __forceinline__ float block_max_f(float v, float* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = dev::warp_max(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  float t = lane < nw ? sh[lane] : 0.0f;
  t = dev::warp_max(t);
  __syncthreads();
  return t;  // every thread
}
__device__ __forceinline__ unsigned block_sum_u(unsigned v, unsigned* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = dev::warp_sum_u(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  unsigned t = lane < nw ? sh[lane] : 0u;
  t = dev::warp_sum_u(t);
  __syncthreads();
  return t;
}
__device__ __forceinline__ dev::f2 block_sum_pair(dev::f2 v, float* shh, float* shl) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = dev::warp_sum_pair(v);
  if (lane == 0) {
    shh[warp] = v.hi;
    shl[warp] = v.lo;
  }
  __syncthreads();
  dev::f2 t = lane < nw ? dev::f2{shh[lane], shl[lane]} : dev::f2{0.0f, 0.0f};
  t = dev::warp_sum_pair(t);
  __syncthreads();
  return t;
}

// Bytes of shared memory an instance needs in warp mode: six state arrays (y_hi, y_lo, x, v_hi,
// v_lo, neighbour sums) and, for a CSR instance, its row offsets and 16-bit local ids; for an
// assignment instance its row and column sums as float pairs.
__host__ __device__ __forceinline__ int warp_bytes(int n, int nnz, int kind) {
  const int base = 4 * 6 * n;
  if (kind == GN_INSTANCE_ASSIGNMENT) {
    const int kk = (int)lrint(sqrt((double)n));
    return base + 16 * kk;
  }
  return base + 4 * (n + 1) + ((2 * nnz + 15) & ~15);
}

// Warp mode: each warp takes instances from the second queue and runs each to its stop test with
// warp synchronisation only.  The per-row arithmetic is the CTA mode's: G lanes per CSR row with
// the same lane split and shuffle order, lane-sequential row and column sums for an assignment
// instance, the same update and the same stop decision (max and count reductions, exact).
__device__ void run_warp_instances(const BatchParams& P, unsigned char* smem) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* wsm = smem + (size_t)warp * (size_t)P.wbytes;
  const float th_lo = (float)P.theta, th_hi = (float)(1.0 - P.theta);
  for (;;) {
    unsigned q = 0;
    if (lane == 0) q = atomicAdd(P.queue + 1, 1u);
    q = __shfl_sync(0xffffffffu, q, 0);
    if (q >= (unsigned)(P.count - P.nbig)) return;
    const int inst = P.order[P.nbig + q];
    const int64_t v0 = P.vtx_off[inst];
    const int n = (int)(P.vtx_off[inst + 1] - v0);
    const int kind = P.kind[inst];
    const int64_t e0 = P.ent_off[inst];
    const int nnz = (int)(P.ent_off[inst + 1] - e0);
    const int32_t* rp_g = P.row_ptr + v0 + inst;
    const int32_t* ci_g = P.col_idx + e0;
    const int kk = kind == GN_INSTANCE_ASSIGNMENT ? (int)lrintf(sqrtf((float)n)) : 0;
    const int G = P.group[inst];
    float* s_yh = reinterpret_cast<float*>(wsm);
    float* s_yl = s_yh + n;
    float* s_x = s_yl + n;
    float* s_vh = s_x + n;
    float* s_vl = s_vh + n;
    float* s_sum = s_vl + n;
    int* s_rp = reinterpret_cast<int*>(s_sum + n);        // CSR
    float* s_rs = s_sum + n;                              // assignment: rh, rl, ch, cl (kk each)
    uint16_t* s_id = reinterpret_cast<uint16_t*>(s_rp + n + 1);
    for (int i = lane; i < n; i += 32) {
      const float xi = P.x[v0 + i];
      const dev::f2 vv = {P.v[v0 + i], P.vlo[v0 + i]};
      const dev::f2 yy = dev::mul_f2(vv, dev::f2{xi, 0.0f});
      s_x[i] = xi;
      s_vh[i] = vv.hi;
      s_vl[i] = vv.lo;
      s_yh[i] = yy.hi;
      s_yl[i] = yy.lo;
    }
    if (kind == GN_INSTANCE_CSR) {
      for (int i = lane; i <= n; i += 32) s_rp[i] = rp_g[i];
      for (int e = lane; e < nnz; e += 32) s_id[e] = (uint16_t)ci_g[e];
    }
    __syncwarp();
    unsigned hits = 0;
    int k = 0, stop = 0;
    float last_r = 0.0f;
    unsigned last_n = 0;
    dev::f2 last_obj = {0.0f, 0.0f};
    float last_l1 = 0.0f, last_en = 0.0f;
    int next_chk = P.check_every;  // a check follows step next_chk - 1
    const int grp = lane / G, gl = lane & (G - 1), ngrp = 32 / G;  // CSR: G lanes per row
    const float inv_kk = kk > 0 ? 1.0f / (float)kk : 0.0f;        // assignment: row of a cell
    for (; k < P.k_end; ++k) {
      const float2 gg = P.gtab[k < P.gtab_len ? k : P.gtab_len - 1];
      const dev::f2 gam = {gg.x, gg.y};
      if (kind == GN_INSTANCE_CSR) {
        for (int base = 0; base < n; base += ngrp) {
          const int r = base + grp;
          float acc = 0.0f;
          if (r < n) {
            const int a = s_rp[r], c = s_rp[r + 1];
            for (int e = a + gl; e < c; e += G) acc += s_yh[s_id[e]];
          }
          for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (r < n && gl == 0) s_sum[r] = acc;
        }
      } else {
        for (int t = lane; t < 2 * kk; t += 32) {
          const bool row = t < kk;
          const int q2 = row ? t : t - kk;
          dev::f2 a = {0.0f, 0.0f};
          for (int j = 0; j < kk; ++j) {
            const float yv = row ? s_yh[q2 * kk + j] : s_yh[j * kk + q2];
            const dev::f2 s = dev::two_sum(a.hi, yv);
            a = dev::fast_two_sum(s.hi, dev::fadd(s.lo, a.lo));
          }
          s_rs[(row ? 0 : 2 * kk) + q2] = a.hi;
          s_rs[(row ? kk : 3 * kk) + q2] = a.lo;
        }
      }
      __syncwarp();
      const bool due = k + 1 == next_chk;
      const bool check = due || (k + 1 == P.k_end);
      if (due) next_chk += P.check_every;
      CheckAcc acc;
      for (int i = lane; i < n; i += 32) {
        Own o = {s_yh[i], s_yl[i], s_x[i]};
        float sn;
        if (kind == GN_INSTANCE_CSR) {
          sn = s_sum[i];
        } else {
          // floor(i / k): (i + 1/2) / k stays 1/(2k) >= 2^-8 from an integer (k <= 128, i < 2^14),
          // far more than the FP32 rounding of the product
          const int r = (int)(((float)i + 0.5f) * inv_kk), c = i - r * kk;
          const float yv = o.pub;
          dev::f2 a = dev::two_sum(s_rs[r], -yv);
          a.lo = dev::fadd(a.lo, s_rs[kk + r]);
          dev::f2 b = dev::two_sum(s_rs[2 * kk + c], -yv);
          b.lo = dev::fadd(b.lo, s_rs[3 * kk + c]);
          const dev::f2 t = dev::two_sum(a.hi, b.hi);
          sn = dev::fadd(t.hi, dev::fadd(t.lo, dev::fadd(a.lo, b.lo)));
        }
        update_one(o, dev::f2{s_vh[i], s_vl[i]}, sn, gam, check, check ? P.w[v0 + i] : 0.0f, th_lo, th_hi, hits,
                   acc);
        s_yh[i] = o.pub;
        s_yl[i] = o.aux;
        s_x[i] = o.xs;
      }
      __syncwarp();
      if (check) {
        const float r = dev::warp_max(acc.rmax);
        const unsigned nb = dev::warp_sum_u(acc.nonbin);
        const dev::f2 ob = dev::warp_sum_f2(acc.obj);
        const dev::f2 dg = dev::two_sum(gg.x, -P.thr_hi);
        const bool bin_ok = nb == 0u && dev::fadd(dg.hi, dev::fadd(dg.lo, dev::fsub(gg.y, P.thr_lo))) > 0.0f;
        const bool res_ok = P.res_test && r <= P.tol_f;
        last_r = r;
        last_n = nb;
        last_obj = ob;
        last_l1 = acc.l1;
        last_en = acc.en;
        if (bin_ok || res_ok) {
          stop = 1;
          ++k;
          break;
        }
      }
    }
    for (int i = lane; i < n; i += 32) P.x[v0 + i] = own_x(Own{s_yh[i], s_yl[i], s_x[i]}, s_vh[i]);
    const dev::f2 l1s = dev::warp_sum_f2(last_l1);
    const dev::f2 ens = dev::warp_sum_f2(last_en);
    const unsigned long long h = dev::warp_sum_ull(hits);
    if (lane == 0) {
      BatchInfoDev bi;
      bi.iters = k;
      bi.converged = stop;
      bi.binary = last_n == 0u;
      bi.nonbin = last_n;
      bi.hits = h;
      bi.resid_inf = last_r;
      bi.pad = 0.0f;
      bi.objective = (double)last_obj.hi + (double)last_obj.lo;
      bi.resid_l1 = (double)l1s.hi + (double)l1s.lo;
      bi.energy = (double)ens.hi + (double)ens.lo;
      P.info[inst] = bi;
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kBatchMaxThreads, 1) k_gn_batch(const BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_inst;
  __shared__ float s_rf[32];
  __shared__ unsigned s_ru[32];
  __shared__ float s_ph[32], s_pl[32];
  const int tid = threadIdx.x, lane = tid & 31;
  // shared memory: [y_hi y_lo x v_hi v_lo (nmax each) | row and column sums as float pairs
  // (assignment, k <= 128) | neighbour sums, row offsets (CSR, ncsr) | local ids (CSR)].
  // Assignment instances form their neighbour sums inside the update, so a k = 96 instance
  // (9216 vertices) fits.
  const int N = P.nmax, NC = P.ncsr;
  float* s_yh = reinterpret_cast<float*>(smem);
  float* s_yl = s_yh + N;
  float* s_x = s_yl + N;
  float* s_vh = s_x + N;
  float* s_vl = s_vh + N;
  float* s_rh = s_vl + N;
  float* s_rl = s_rh + 128;
  float* s_ch = s_rl + 128;
  float* s_cl = s_ch + 128;
  float* s_sum = s_cl + 128;
  int* s_rp = reinterpret_cast<int*>(s_sum + NC);
  uint16_t* s_id = reinterpret_cast<uint16_t*>(s_rp + NC + 4);
  const float th_lo = (float)P.theta, th_hi = (float)(1.0 - P.theta);

  for (;;) {
    if (tid == 0) {
      const unsigned q = atomicAdd(P.queue, 1u);
      s_inst = q < (unsigned)P.nbig ? P.order[q] : -1;
    }
    __syncthreads();
    const int inst = s_inst;
    __syncthreads();
    if (inst < 0) break;
    const int64_t v0 = P.vtx_off[inst];
    const int n = (int)(P.vtx_off[inst + 1] - v0);
    const int kind = P.kind[inst];
    const int64_t e0 = P.ent_off[inst];
    const int nnz = (int)(P.ent_off[inst + 1] - e0);
    const int32_t* rp_g = P.row_ptr + v0 + inst;
    const int32_t* ci_g = P.col_idx + e0;
    const bool ids_smem = nnz <= P.idcap;
    int kk = 0;
    if (kind == GN_INSTANCE_ASSIGNMENT) kk = (int)lrintf(sqrtf((float)n));
    const int G = P.group[inst];

    for (int i = tid; i < n; i += blockDim.x) {
      const float xi = P.x[v0 + i];
      const dev::f2 vv = {P.v[v0 + i], P.vlo[v0 + i]};
      const dev::f2 yy = dev::mul_f2(vv, dev::f2{xi, 0.0f});
      s_x[i] = xi;
      s_vh[i] = vv.hi;
      s_vl[i] = vv.lo;
      s_yh[i] = yy.hi;
      s_yl[i] = yy.lo;
    }
    if (kind == GN_INSTANCE_CSR) {
      for (int i = tid; i <= n; i += blockDim.x) s_rp[i] = rp_g[i];
      if (ids_smem)
        for (int e = tid; e < nnz; e += blockDim.x) s_id[e] = (uint16_t)ci_g[e];
    }
    __syncthreads();

    unsigned hits = 0;
    int k = 0, stop = 0;
    float last_r = 0.0f;
    unsigned last_n = 0;
    dev::f2 last_obj = {0.0f, 0.0f};
    float last_l1 = 0.0f, last_en = 0.0f;  // this thread's terms at the last check
    int next_chk = P.check_every;  // a check follows step next_chk - 1
    const int grp = tid / G, gl = tid & (G - 1), ngrp = blockDim.x / G;  // CSR: G lanes per row
    const float inv_kk = kk > 0 ? 1.0f / (float)kk : 0.0f;                 // assignment: row of a cell
    for (; k < P.k_end; ++k) {
      const float2 gg = P.gtab[k < P.gtab_len ? k : P.gtab_len - 1];
      const dev::f2 gam = {gg.x, gg.y};
      // ---- neighbour sums
      if (kind == GN_INSTANCE_CSR) {
        for (int base = 0; base < n; base += ngrp) {
          const int r = base + grp;
          float acc = 0.0f;
          if (r < n) {
            const int a = s_rp[r], c = s_rp[r + 1];
            if (ids_smem) {
              for (int e = a + gl; e < c; e += G) acc += s_yh[s_id[e]];
            } else {
              for (int e = a + gl; e < c; e += G) acc += s_yh[ci_g[e]];
            }
          }
          for (int o = G >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (r < n && gl == 0) s_sum[r] = acc;
        }
      } else {
        // row sums (r < kk) and column sums (kk <= t < 2 kk), compensated
        for (int t = tid; t < 2 * kk; t += blockDim.x) {
          const bool row = t < kk;
          const int q = row ? t : t - kk;
          dev::f2 a = {0.0f, 0.0f};
          for (int j = 0; j < kk; ++j) {
            const float yv = row ? s_yh[q * kk + j] : s_yh[j * kk + q];
            const dev::f2 s = dev::two_sum(a.hi, yv);
            a = dev::fast_two_sum(s.hi, dev::fadd(s.lo, a.lo));
          }
          if (row) { s_rh[q] = a.hi; s_rl[q] = a.lo; } else { s_ch[q] = a.hi; s_cl[q] = a.lo; }
        }
      }
      __syncthreads();
      // ---- update (assignment: the neighbour sum from the row and column sums, here)
      const bool due = k + 1 == next_chk;
      const bool check = due || (k + 1 == P.k_end);
      if (due) next_chk += P.check_every;
      CheckAcc acc;
      for (int i = tid; i < n; i += blockDim.x) {
        Own o = {s_yh[i], s_yl[i], s_x[i]};
        float sn;
        if (kind == GN_INSTANCE_CSR) {
          sn = s_sum[i];
        } else {
          // floor(i / k): (i + 1/2) / k stays 1/(2k) >= 2^-8 from an integer (k <= 128, i < 2^14),
          // far more than the FP32 rounding of the product
          const int r = (int)(((float)i + 0.5f) * inv_kk), c = i - r * kk;
          const float yv = o.pub;
          // (R_r - y) + (C_c - y) in float pairs
          dev::f2 a = dev::two_sum(s_rh[r], -yv);
          a.lo = dev::fadd(a.lo, s_rl[r]);
          dev::f2 b = dev::two_sum(s_ch[c], -yv);
          b.lo = dev::fadd(b.lo, s_cl[c]);
          const dev::f2 t = dev::two_sum(a.hi, b.hi);
          sn = dev::fadd(t.hi, dev::fadd(t.lo, dev::fadd(a.lo, b.lo)));
        }
        update_one(o, dev::f2{s_vh[i], s_vl[i]}, sn, gam, check, check ? P.w[v0 + i] : 0.0f, th_lo, th_hi, hits,
                   acc);
        s_yh[i] = o.pub;
        s_yl[i] = o.aux;
        s_x[i] = o.xs;
      }
      __syncthreads();
      if (check) {
        const float r = block_max_f(acc.rmax, s_rf);
        const unsigned nb = block_sum_u(acc.nonbin, s_ru);
        const dev::f2 ob = block_sum_pair(dev::f2{acc.obj, 0.0f}, s_ph, s_pl);
        const dev::f2 dg = dev::two_sum(gg.x, -P.thr_hi);
        const bool bin_ok = nb == 0u && dev::fadd(dg.hi, dev::fadd(dg.lo, dev::fsub(gg.y, P.thr_lo))) > 0.0f;
        const bool res_ok = P.res_test && r <= P.tol_f;
        last_r = r;
        last_n = nb;
        last_obj = ob;
        last_l1 = acc.l1;
        last_en = acc.en;
        if (bin_ok || res_ok) {
          stop = 1;
          ++k;
          break;
        }
      }
    }
    // ---- results (the last check's residual sum and energy: summed once, here)
    for (int i = tid; i < n; i += blockDim.x) P.x[v0 + i] = own_x(Own{s_yh[i], s_yl[i], s_x[i]}, s_vh[i]);
    const dev::f2 l1s = block_sum_pair(dev::f2{last_l1, 0.0f}, s_ph, s_pl);
    const dev::f2 ens = block_sum_pair(dev::f2{last_en, 0.0f}, s_ph, s_pl);
    unsigned long long h = dev::warp_sum_ull(hits);
    __shared__ unsigned long long s_h[32];
    if (lane == 0) s_h[tid >> 5] = h;
    __syncthreads();
    if (tid == 0) {
      unsigned long long t = 0;
      for (int j = 0; j < (int)(blockDim.x >> 5); ++j) t += s_h[j];
      BatchInfoDev bi;
      bi.iters = k;
      bi.converged = stop;
      bi.binary = last_n == 0u;
      bi.nonbin = last_n;
      bi.hits = t;
      bi.resid_inf = last_r;
      bi.pad = 0.0f;
      bi.objective = (double)last_obj.hi + (double)last_obj.lo;
      bi.resid_l1 = (double)l1s.hi + (double)l1s.lo;
      bi.energy = (double)ens.hi + (double)ens.lo;
      P.info[inst] = bi;
    }
    __syncthreads();
  }
  // warp mode for the small instances
  if (P.nbig < P.count) run_warp_instances(P, smem);
}

// ---- validation and preparation kernels (thread per global vertex)

__device__ __forceinline__ int find_instance(const int64_t* off, int count, int64_t g) {
  int lo = 0, hi = count;  // off[lo] <= g < off[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= g) lo = mid; else hi = mid;
  }
  return lo;
}

__global__ void k_batch_check(int count, int64_t ntot, const int64_t* __restrict__ vtx_off,
                              const int64_t* __restrict__ ent_off, const int32_t* __restrict__ rp,
                              const int32_t* __restrict__ ci, const int32_t* __restrict__ kind,
                              const float* __restrict__ w, float* __restrict__ v, float* __restrict__ vlo,
                              int* flags) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntot) return;
  const int inst = find_instance(vtx_off, count, g);
  const int64_t v0 = vtx_off[inst];
  const int n = (int)(vtx_off[inst + 1] - v0);
  const int i = (int)(g - v0);
  const float wi = w[g];
  dev::f2 vv = {1.0f, 0.0f};
  if (!(wi > 0.0f) || !isfinite(wi)) atomicOr(flags, DEV_BAD_WEIGHT);
  else vv = dev::split_f64(sqrt((double)wi));
  v[g] = vv.hi;
  vlo[g] = vv.lo;
  if (kind[inst] != GN_INSTANCE_CSR) return;
  const int32_t* r = rp + v0 + inst;
  const int nnz = (int)(ent_off[inst + 1] - ent_off[inst]);
  const int a = r[i], b = r[i + 1];
  if ((i == 0 && a != 0) || b < a || b > nnz || (i == n - 1 && b != nnz)) {
    atomicOr(flags, DEV_BAD_CSR);
    return;
  }
  const int32_t* c = ci + ent_off[inst];
  int prev = -1;
  for (int e = a; e < b; ++e) {
    const int j = c[e];
    if (j < 0 || j >= n) {
      atomicOr(flags, DEV_BAD_CSR);
      return;
    }
    if (j == i || j <= prev) atomicOr(flags, DEV_NOT_SIMPLE);
    prev = j;
  }
}

__global__ void k_batch_symmetry(int count, int64_t ntot, const int64_t* __restrict__ vtx_off,
                                 const int64_t* __restrict__ ent_off, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, const int32_t* __restrict__ kind, int* flags) {
  if (dev::ld_relaxed_int(flags) & DEV_BAD_CSR) return;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntot) return;
  const int inst = find_instance(vtx_off, count, g);
  if (kind[inst] != GN_INSTANCE_CSR) return;
  const int64_t v0 = vtx_off[inst];
  const int i = (int)(g - v0);
  const int32_t* r = rp + v0 + inst;
  const int32_t* c = ci + ent_off[inst];
  for (int e = r[i]; e < r[i + 1]; ++e) {
    const int j = c[e];
    int a = r[j], b = r[j + 1] - 1;
    bool found = false;
    while (a <= b) {
      const int m = (a + b) >> 1;
      if (c[m] == i) { found = true; break; }
      if (c[m] < i) a = m + 1; else b = m - 1;
    }
    if (!found) {
      atomicOr(flags, DEV_NOT_SIMPLE);
      return;
    }
  }
}

// start state x0 (or 1/(deg+1)) and the normalizability check of Def. 1
__global__ void k_batch_init(int count, int64_t ntot, const int64_t* __restrict__ vtx_off,
                             const int64_t* __restrict__ ent_off, const int32_t* __restrict__ rp,
                             const int32_t* __restrict__ ci, const int32_t* __restrict__ kind,
                             const float* __restrict__ x0, float* __restrict__ x, int* flags) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= ntot) return;
  const int inst = find_instance(vtx_off, count, g);
  const int64_t v0 = vtx_off[inst];
  const int n = (int)(vtx_off[inst + 1] - v0);
  const int i = (int)(g - v0);
  int deg;
  if (kind[inst] == GN_INSTANCE_CSR) {
    const int32_t* r = rp + v0 + inst;
    deg = r[i + 1] - r[i];
  } else {
    const int kk = (int)lrintf(sqrtf((float)n));
    deg = 2 * (kk - 1);
  }
  float xi = x0 ? x0[g] : __frcp_rn((float)(deg + 1));
  bool bad = !(xi >= 0.0f) || !isfinite(xi);
  if (x0 && !bad && !(xi > 0.0f)) {
    bool pos = false;
    if (kind[inst] == GN_INSTANCE_CSR) {
      const int32_t* r = rp + v0 + inst;
      const int32_t* c = ci + ent_off[inst];
      for (int e = r[i]; e < r[i + 1] && !pos; ++e) pos = x0[v0 + c[e]] > 0.0f;
    } else {
      const int kk = (int)lrintf(sqrtf((float)n));
      const int rr = i / kk, cc = i - rr * kk;
      for (int j = 0; j < kk && !pos; ++j)
        pos = (j != cc && x0[v0 + rr * kk + j] > 0.0f) || (j != rr && x0[v0 + j * kk + cc] > 0.0f);
    }
    bad = !pos;
  }
  if (bad) atomicOr(flags, DEV_NOT_NORMALIZABLE);
  x[g] = xi;
}

__global__ void k_batch_gamma(int len, int mode, double g0, double g1, int T, float2* __restrict__ out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= len) return;
  const dev::f2 p = dev::split_f64(dev::gamma_at(mode, g0, g1, T, k));
  out[k] = make_float2(p.hi, p.lo);
}

// extraction per instance: CTA per instance; rounding, exact independence and maximality,
// count and W(S) (float-pair sums, FP64 result)
__global__ void k_batch_extract(int count, const int64_t* __restrict__ vtx_off, const int64_t* __restrict__ ent_off,
                                const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                                const int32_t* __restrict__ kind, const float* __restrict__ x,
                                const float* __restrict__ w, uint8_t* __restrict__ mask,
                                int* __restrict__ out_status, int* __restrict__ out_count,
                                double* __restrict__ out_weight) {
  __shared__ int s_indep, s_maxi;
  __shared__ unsigned s_ru[32];
  __shared__ float s_ph[32], s_pl[32];
  const int inst = blockIdx.x;
  if (inst >= count) return;
  const int64_t v0 = vtx_off[inst];
  const int n = (int)(vtx_off[inst + 1] - v0);
  if (threadIdx.x == 0) {
    s_indep = 1;
    s_maxi = 1;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) mask[v0 + i] = x[v0 + i] > 0.5f ? 1 : 0;
  __syncthreads();
  unsigned cnt = 0;
  float wsum = 0.0f, wlo = 0.0f;
  const bool csr = kind[inst] == GN_INSTANCE_CSR;
  const int kk = csr ? 0 : (int)lrintf(sqrtf((float)n));
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const bool in = mask[v0 + i] != 0;
    bool covered = false, clash = false;
    if (csr) {
      const int32_t* r = rp + v0 + inst;
      const int32_t* c = ci + ent_off[inst];
      for (int e = r[i]; e < r[i + 1]; ++e)
        if (mask[v0 + c[e]]) { covered = true; if (in) clash = true; }
    } else {
      const int rr = i / kk, cc = i - rr * kk;
      for (int j = 0; j < kk; ++j) {
        if (j != cc && mask[v0 + rr * kk + j]) { covered = true; if (in) clash = true; }
        if (j != rr && mask[v0 + j * kk + cc]) { covered = true; if (in) clash = true; }
      }
    }
    if (clash) s_indep = 0;
    if (!in && !covered) s_maxi = 0;
    if (in) {
      ++cnt;
      const dev::f2 s = dev::two_sum(wsum, w[v0 + i]);
      wsum = s.hi;
      wlo = dev::fadd(wlo, s.lo);
    }
  }
  const unsigned tc = block_sum_u(cnt, s_ru);
  const dev::f2 tw = block_sum_pair(dev::fast_two_sum(wsum, wlo), s_ph, s_pl);
  if (threadIdx.x == 0) {
    out_count[inst] = (int)tc;
    out_weight[inst] = (double)tw.hi + (double)tw.lo;
    out_status[inst] = !s_indep ? GN_ERR_NOT_INDEPENDENT : (!s_maxi ? GN_WARN_NOT_MAXIMAL : GN_OK);
  }
}

}  // namespace gn

// ------------------------------------------------------------------------------------------
// handle

struct gn_batch {
  int device = 0, num_sms = 0, io_mem = GN_HOST;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int count = 0;
  int64_t ntot = 0, etot = 0;
  int nmax = 0;
  int ncsr = 0;
  int64_t* d_vtx_off = nullptr;
  int64_t* d_ent_off = nullptr;
  int32_t* d_rp = nullptr;
  int32_t* d_ci = nullptr;
  int32_t* d_kind = nullptr;
  int32_t* d_order = nullptr;
  int32_t* d_group = nullptr;
  float* d_w = nullptr;
  float* d_v = nullptr;
  float* d_vlo = nullptr;
  float* d_x = nullptr;
  float* d_io = nullptr;
  gn::BatchInfoDev* d_info = nullptr;
  gn::BatchInfoDev* h_info = nullptr;   // pinned
  unsigned* d_queue = nullptr;
  int* d_flags = nullptr;
  int* h_flags = nullptr;               // pinned
  float2* d_gtab = nullptr;
  int gtab_cap = 0;
  uint8_t* d_mask = nullptr;
  int* d_xstatus = nullptr;
  int* d_xcount = nullptr;
  double* d_xweight = nullptr;
  std::vector<int64_t> h_vtx_off;
  int threads = 512;                    // CTA size (autotuned)
  int ctas = 0;
  int idcap = 0;
  size_t smem = 0;
  int wmax = 0;                         // instances up to this many vertices run a warp each (0: none)
  int wbytes = 0;                       // shared memory of one warp in warp mode
  int nbig = 0;                         // instances in CTA mode (the rest: warp mode)
  std::vector<double> h_work;           // per instance: work estimate, size, entries, kind
  std::vector<int> h_n, h_e, h_kind;
  // captured run
  cudaGraphExec_t graph = nullptr;
  struct Key {
    int max_iters = -1;
    double tol = 0;
    gn_params p;
    const float* x0 = nullptr;
    int threads = 0;
  } key;
  bool has_state = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

namespace gn {

// the processing order: CTA-mode instances by decreasing work, then the warp-mode ones (at most
// wmax vertices and fitting one warp's share of shared memory) by decreasing work
static gn_status batch_order(gn_batch* b) {
  std::vector<int32_t> big, small;
  for (int i = 0; i < b->count; ++i) {
    const bool w = b->wmax > 0 && b->h_n[i] <= b->wmax && warp_bytes(b->h_n[i], b->h_e[i], b->h_kind[i]) <= b->wbytes;
    (w ? small : big).push_back(i);
  }
  auto by_work = [&](int a, int c) { return b->h_work[a] > b->h_work[c]; };
  std::stable_sort(big.begin(), big.end(), by_work);
  std::stable_sort(small.begin(), small.end(), by_work);
  b->nbig = (int)big.size();
  big.insert(big.end(), small.begin(), small.end());
  if (b->count > 0)
    GN_CUDA(cudaMemcpyAsync(b->d_order, big.data(), sizeof(int32_t) * b->count, cudaMemcpyHostToDevice, b->stream));
  GN_CUDA(cudaStreamSynchronize(b->stream));
  return GN_OK;
}

static size_t batch_smem(int nmax, int ncsr, int idcap) {
  return sizeof(float) * (5 * (size_t)nmax + 4 * 128 + (size_t)ncsr) + sizeof(int) * ((size_t)ncsr + 4) +
         sizeof(uint16_t) * (size_t)idcap;
}

// CTA size -> CTAs per SM and the id capacity that still fits
static gn_status batch_config(gn_batch* b, int threads) {
  const size_t base = batch_smem(b->nmax, b->ncsr, 0);
  const size_t limit = 220 * 1024;
  if (base > limit) return fail(GN_ERR_TOO_LARGE, "gn_batch: largest instance exceeds shared memory");
  // prefer two CTAs per SM for 512 threads or fewer when the base layout allows it
  int per_sm_target = threads <= 512 ? 2 : 1;
  size_t budget = limit / per_sm_target;
  if (base > budget) {
    per_sm_target = 1;
    budget = limit;
  }
  const int idcap = (int)std::min<size_t>((budget - base) / sizeof(uint16_t), 1 << 20);
  const size_t smem = batch_smem(b->nmax, b->ncsr, idcap);
  GN_CUDA(cudaFuncSetAttribute((const void*)k_gn_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)limit));
  int per_sm = 0;
  GN_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gn_batch, threads, smem));
  if (per_sm < 1) return fail(GN_ERR_TOO_LARGE, "gn_batch: kernel does not fit an SM");
  b->threads = threads;
  b->idcap = idcap;
  b->smem = smem;
  b->ctas = std::min<int64_t>((int64_t)per_sm * b->num_sms, std::max(1, b->count));
  b->wbytes = (int)((smem / (size_t)(threads / 32)) & ~(size_t)15);
  return batch_order(b);
}

}  // namespace gn

extern "C" void gn_batch_destroy(gn_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  if (b->stream) cudaStreamSynchronize(b->stream);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  void* d[] = {b->d_vtx_off, b->d_ent_off, b->d_rp, b->d_ci, b->d_kind, b->d_order, b->d_group, b->d_w,
               b->d_v, b->d_vlo, b->d_x, b->d_io, b->d_info, b->d_queue, b->d_flags, b->d_gtab, b->d_mask,
               b->d_xstatus, b->d_xcount, b->d_xweight};
  for (void* p : d)
    if (p) cudaFree(p);
  if (b->h_info) cudaFreeHost(b->h_info);
  if (b->h_flags) cudaFreeHost(b->h_flags);
  if (b->ev0) cudaEventDestroy(b->ev0);
  if (b->ev1) cudaEventDestroy(b->ev1);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

extern "C" gn_status gn_batch_create(gn_batch** out, int32_t count, const int64_t* vtx_off,
                                     const int64_t* ent_off, const int32_t* row_ptr,
                                     const int32_t* col_idx, const float* w, const int32_t* kind,
                                     int mem, void* stream) {
  using namespace gn;
  if (!out) return fail(GN_ERR_ARG, "gn_batch_create: out is NULL");
  *out = nullptr;
  if (count < 0 || !vtx_off || !ent_off || (mem != GN_HOST && mem != GN_DEVICE))
    return fail(GN_ERR_ARG, "gn_batch_create: bad argument");
  gn_batch* b = new gn_batch();
  struct Guard {
    gn_batch*& b;
    ~Guard() { if (b) gn_batch_destroy(b); }
  } guard{b};
  b->io_mem = mem;
  b->count = count;
  GN_CUDA(cudaGetDevice(&b->device));
  GN_CUDA(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, b->device));
  if (stream) {
    b->stream = (cudaStream_t)stream;
  } else {
    GN_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    b->own_stream = true;
  }
  // offsets and kinds on the host (size checks, work order)
  std::vector<int64_t> vo(count + 1), eo(count + 1);
  std::vector<int32_t> kd(std::max(count, 1), GN_INSTANCE_CSR);
  cudaMemcpyKind k2h = mem == GN_HOST ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost;
  GN_CUDA(cudaMemcpy(vo.data(), vtx_off, sizeof(int64_t) * (count + 1), k2h));
  GN_CUDA(cudaMemcpy(eo.data(), ent_off, sizeof(int64_t) * (count + 1), k2h));
  if (kind && count > 0) GN_CUDA(cudaMemcpy(kd.data(), kind, sizeof(int32_t) * count, k2h));
  if (vo[0] != 0 || eo[0] != 0) return fail(GN_ERR_ARG, "gn_batch_create: offsets must start at 0");
  std::vector<double> work(std::max(count, 1));
  std::vector<int32_t> grp(std::max(count, 1), 1);
  for (int i = 0; i < count; ++i) {
    const int64_t n = vo[i + 1] - vo[i], e = eo[i + 1] - eo[i];
    if (n < 1 || e < 0) return fail(GN_ERR_ARG, "gn_batch_create: empty instance or decreasing offsets");
    if (n > 16384) return fail(GN_ERR_TOO_LARGE, "gn_batch_create: instances are limited to 16384 vertices");
    if (kd[i] == GN_INSTANCE_ASSIGNMENT) {
      const int64_t kk = (int64_t)std::llround(std::sqrt((double)n));
      if (kk * kk != n || kk > 128 || e != 0)
        return fail(GN_ERR_ARG, "gn_batch_create: an assignment instance needs n = k*k, k <= 128, no entries");
      work[i] = (double)n * 4;
    } else if (kd[i] == GN_INSTANCE_CSR) {
      work[i] = (double)e + 4.0 * n;
      int G = 1;
      const double avg = (double)e / n;
      while (G < 32 && G * 3 < avg) G <<= 1;
      grp[i] = G;
      b->ncsr = std::max<int>(b->ncsr, (int)n);
    } else {
      return fail(GN_ERR_ARG, "gn_batch_create: unknown instance kind");
    }
    b->nmax = std::max<int>(b->nmax, (int)n);
  }
  b->ntot = vo[count];
  b->etot = eo[count];
  b->h_vtx_off = vo;
  b->h_work = work;
  b->h_n.resize(count);
  b->h_e.resize(count);
  b->h_kind.assign(kd.begin(), kd.begin() + count);
  for (int i = 0; i < count; ++i) {
    b->h_n[i] = (int)(vo[i + 1] - vo[i]);
    b->h_e[i] = (int)(eo[i + 1] - eo[i]);
  }

  const size_t nv = (size_t)std::max<int64_t>(b->ntot, 1);
  GN_CUDA(cudaMalloc(&b->d_vtx_off, sizeof(int64_t) * (count + 1)));
  GN_CUDA(cudaMalloc(&b->d_ent_off, sizeof(int64_t) * (count + 1)));
  GN_CUDA(cudaMalloc(&b->d_rp, sizeof(int32_t) * (nv + count + 1)));
  GN_CUDA(cudaMalloc(&b->d_ci, sizeof(int32_t) * (size_t)std::max<int64_t>(b->etot, 1)));
  GN_CUDA(cudaMalloc(&b->d_kind, sizeof(int32_t) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_order, sizeof(int32_t) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_group, sizeof(int32_t) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_w, sizeof(float) * nv));
  GN_CUDA(cudaMalloc(&b->d_v, sizeof(float) * nv));
  GN_CUDA(cudaMalloc(&b->d_vlo, sizeof(float) * nv));
  GN_CUDA(cudaMalloc(&b->d_x, sizeof(float) * nv));
  GN_CUDA(cudaMalloc(&b->d_io, sizeof(float) * nv));
  GN_CUDA(cudaMalloc(&b->d_info, sizeof(BatchInfoDev) * std::max(count, 1)));
  GN_CUDA(cudaMallocHost(&b->h_info, sizeof(BatchInfoDev) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_queue, sizeof(unsigned) * 4));
  GN_CUDA(cudaMalloc(&b->d_flags, sizeof(int) * 4));
  GN_CUDA(cudaMallocHost(&b->h_flags, sizeof(int) * 4));
  GN_CUDA(cudaMalloc(&b->d_mask, nv));
  GN_CUDA(cudaMalloc(&b->d_xstatus, sizeof(int) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_xcount, sizeof(int) * std::max(count, 1)));
  GN_CUDA(cudaMalloc(&b->d_xweight, sizeof(double) * std::max(count, 1)));
  GN_CUDA(cudaEventCreate(&b->ev0));
  GN_CUDA(cudaEventCreate(&b->ev1));
  cudaMemcpyKind kin = mem == GN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GN_CUDA(cudaMemcpyAsync(b->d_vtx_off, vo.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, b->stream));
  GN_CUDA(cudaMemcpyAsync(b->d_ent_off, eo.data(), sizeof(int64_t) * (count + 1), cudaMemcpyHostToDevice, b->stream));
  GN_CUDA(cudaMemcpyAsync(b->d_kind, kd.data(), sizeof(int32_t) * std::max(count, 1), cudaMemcpyHostToDevice, b->stream));
  GN_CUDA(cudaMemcpyAsync(b->d_group, grp.data(), sizeof(int32_t) * std::max(count, 1), cudaMemcpyHostToDevice, b->stream));
  if (b->ntot > 0) {
    if (!w) return fail(GN_ERR_ARG, "gn_batch_create: w is NULL");
    GN_CUDA(cudaMemcpyAsync(b->d_w, w, sizeof(float) * b->ntot, kin, b->stream));
    if (row_ptr) GN_CUDA(cudaMemcpyAsync(b->d_rp, row_ptr, sizeof(int32_t) * (b->ntot + count), kin, b->stream));
    else GN_CUDA(cudaMemsetAsync(b->d_rp, 0, sizeof(int32_t) * (b->ntot + count), b->stream));
  }
  if (b->etot > 0) {
    if (!col_idx || !row_ptr) return fail(GN_ERR_ARG, "gn_batch_create: col_idx or row_ptr is NULL");
    GN_CUDA(cudaMemcpyAsync(b->d_ci, col_idx, sizeof(int32_t) * b->etot, kin, b->stream));
  }
  GN_CUDA(cudaMemsetAsync(b->d_flags, 0, sizeof(int) * 4, b->stream));
  if (b->ntot > 0) {
    const unsigned grid = (unsigned)((b->ntot + 255) / 256);
    k_batch_check<<<grid, 256, 0, b->stream>>>(count, b->ntot, b->d_vtx_off, b->d_ent_off, b->d_rp, b->d_ci,
                                                b->d_kind, b->d_w, b->d_v, b->d_vlo, b->d_flags);
    GN_LAUNCHED();
    k_batch_symmetry<<<grid, 256, 0, b->stream>>>(count, b->ntot, b->d_vtx_off, b->d_ent_off, b->d_rp, b->d_ci,
                                                   b->d_kind, b->d_flags);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
  }
  GN_CUDA(cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  GN_CUDA(cudaStreamSynchronize(b->stream));
  if (b->h_flags[0] & DEV_BAD_CSR) return fail(GN_ERR_ARG, "gn_batch_create: malformed CSR");
  if (b->h_flags[0] & DEV_NOT_SIMPLE) return fail(GN_ERR_NOT_SIMPLE, "gn_batch_create: an instance is not simple");
  if (b->h_flags[0] & DEV_BAD_WEIGHT) return fail(GN_ERR_WEIGHT, "gn_batch_create: weight <= 0 or not finite");
  gn_status st = batch_config(b, 512);
  if (st != GN_OK) return st;
  *out = b;
  b = nullptr;
  return GN_OK;
}

extern "C" gn_status gn_batch_set_threads(gn_batch* b, int threads) {
  using namespace gn;
  if (!b || (threads != 128 && threads != 256 && threads != 512 && threads != 1024))
    return fail(GN_ERR_ARG, "gn_batch_set_threads: threads must be 128, 256, 512 or 1024");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return batch_config(b, threads);
}

extern "C" gn_status gn_batch_set_packing(gn_batch* b, int warp_max_vertices) {
  using namespace gn;
  if (!b || warp_max_vertices < 0) return fail(GN_ERR_ARG, "gn_batch_set_packing: bad argument");
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->wmax = warp_max_vertices;
  return batch_order(b);
}

extern "C" gn_status gn_batch_packing(const gn_batch* b, int* warp_max_vertices, int* warp_instances) {
  if (!b) return gn::fail(GN_ERR_ARG, "gn_batch_packing: NULL handle");
  if (warp_max_vertices) *warp_max_vertices = b->wmax;
  if (warp_instances) *warp_instances = b->count - b->nbig;
  return GN_OK;
}

namespace gn {

// the run sequence on the handle's stream (captured into a graph by gn_batch_run)
static gn_status batch_enqueue(gn_batch* b, const float* x0_dev, int max_iters, double tol, const gn_params& p) {
  const int glen = (p.gamma_mode == GN_GAMMA_FIXED || p.ramp_iters <= 1) ? 1 : std::max(1, std::min(max_iters, p.ramp_iters));
  GN_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(unsigned) * 2, b->stream));  // CTA and warp queues
  GN_CUDA(cudaMemsetAsync(b->d_flags, 0, sizeof(int) * 4, b->stream));
  k_batch_gamma<<<(glen + 255) / 256, 256, 0, b->stream>>>(glen, p.gamma_mode, p.gamma0, p.gamma1, p.ramp_iters,
                                                          b->d_gtab);
  GN_LAUNCHED();
  const unsigned grid = (unsigned)((b->ntot + 255) / 256);
  k_batch_init<<<grid, 256, 0, b->stream>>>(b->count, b->ntot, b->d_vtx_off, b->d_ent_off, b->d_rp, b->d_ci,
                                             b->d_kind, x0_dev, b->d_x, b->d_flags);
  GN_LAUNCHED();
  BatchParams P;
  P.count = b->count;
  P.vtx_off = b->d_vtx_off;
  P.ent_off = b->d_ent_off;
  P.row_ptr = b->d_rp;
  P.col_idx = b->d_ci;
  P.kind = b->d_kind;
  P.order = b->d_order;
  P.group = b->d_group;
  P.w = b->d_w;
  P.v = b->d_v;
  P.vlo = b->d_vlo;
  P.x = b->d_x;
  P.info = b->d_info;
  P.queue = b->d_queue;
  P.gtab = b->d_gtab;
  P.gtab_len = glen;
  P.k_end = max_iters;
  P.check_every = p.check_every;
  P.theta = p.theta_bin;
  P.tol = tol;
  {
    const double thr = p.theta_bin / (1.0 - p.theta_bin);
    P.thr_hi = (float)thr;
    P.thr_lo = (float)(thr - (double)P.thr_hi);
    P.res_test = tol >= 0.0 ? 1 : 0;
    float f = (float)tol;
    if ((double)f > tol) f = std::nextafter(f, -INFINITY);
    P.tol_f = f;
  }
  P.nmax = b->nmax;
  P.ncsr = b->ncsr;
  P.idcap = b->idcap;
  P.nbig = b->nbig;
  P.wbytes = b->wbytes;
  k_gn_batch<<<b->ctas, b->threads, b->smem, b->stream>>>(P);
  GN_LAUNCHED();
  GN_CUDA(cudaMemcpyAsync(b->h_info, b->d_info, sizeof(BatchInfoDev) * b->count, cudaMemcpyDeviceToHost, b->stream));
  GN_CUDA(cudaMemcpyAsync(b->h_flags, b->d_flags, sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  GN_CUDA(cudaGetLastError());
  return GN_OK;
}

}  // namespace gn

extern "C" gn_status gn_batch_run(gn_batch* b, const float* x0, int max_iters, double tol, const gn_params* pin,
                                  float* x_out, gn_batch_info* info) {
  using namespace gn;
  if (!b) return fail(GN_ERR_ARG, "gn_batch_run: NULL handle");
  gn_params p;
  if (pin) p = *pin; else gn_default_params(&p);
  if (max_iters < 0 || p.check_every < 1 || !(p.theta_bin < 0.5) || p.resume ||
      (p.gamma_mode != GN_GAMMA_PURSUIT && p.gamma_mode != GN_GAMMA_FIXED))
    return fail(GN_ERR_ARG, "gn_batch_run: bad argument");
  GN_CUDA(cudaSetDevice(b->device));
  if (b->count == 0) return GN_OK;
  const int glen = (p.gamma_mode == GN_GAMMA_FIXED || p.ramp_iters <= 1) ? 1 : std::max(1, std::min(max_iters, p.ramp_iters));
  if (glen > b->gtab_cap) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    if (b->d_gtab) cudaFree(b->d_gtab);
    b->d_gtab = nullptr;
    GN_CUDA(cudaMalloc(&b->d_gtab, sizeof(float2) * glen));
    b->gtab_cap = glen;
  }
  const float* x0_dev = nullptr;
  if (x0) {
    if (b->io_mem == GN_DEVICE) {
      x0_dev = x0;
    } else {
      GN_CUDA(cudaMemcpyAsync(b->d_io, x0, sizeof(float) * b->ntot, cudaMemcpyHostToDevice, b->stream));
      x0_dev = b->d_io;
    }
  }
  // the captured sequence is reused while the arguments that shape it are unchanged
  const bool same = b->graph && b->key.max_iters == max_iters && b->key.tol == tol && b->key.x0 == x0_dev &&
                    b->key.threads == b->threads && memcmp(&b->key.p, &p, sizeof p) == 0;
  if (!same) {
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    cudaGraph_t graph = nullptr;
    GN_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    gn_status st = batch_enqueue(b, x0_dev, max_iters, tol, p);
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (st != GN_OK) {
      if (graph) cudaGraphDestroy(graph);
      return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    b->key.max_iters = max_iters;
    b->key.tol = tol;
    b->key.p = p;
    b->key.x0 = x0_dev;
    b->key.threads = b->threads;
  }
  GN_CUDA(cudaEventRecord(b->ev0, b->stream));
  GN_CUDA(cudaGraphLaunch(b->graph, b->stream));
  GN_CUDA(cudaEventRecord(b->ev1, b->stream));
  GN_CUDA(cudaStreamSynchronize(b->stream));
  if (b->h_flags[0] & DEV_NOT_NORMALIZABLE)
    return fail(GN_ERR_NOT_NORMALIZABLE, "gn_batch_run: an x0 is negative, not finite or not normalizable");
  b->has_state = true;
  if (x_out) {
    GN_CUDA(cudaMemcpyAsync(x_out, b->d_x, sizeof(float) * b->ntot,
                            b->io_mem == GN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
    GN_CUDA(cudaStreamSynchronize(b->stream));
  }
  int worst = GN_OK;
  for (int i = 0; i < b->count; ++i) {
    const BatchInfoDev& d = b->h_info[i];
    int st;
    if (!d.converged) st = GN_WARN_NOT_CONVERGED;
    else st = (d.nonbin == 0) ? GN_OK : GN_WARN_NOT_BINARY;
    if (st > worst) worst = st;
    if (info) {
      info[i].iters = d.iters;
      info[i].status = st;
      info[i].converged = d.converged;
      info[i].binary = d.binary;
      info[i].resid_inf = d.resid_inf;
      info[i].objective = d.objective;
      info[i].safe_div_hits = (long long)d.hits;
      info[i].resid_l1 = d.resid_l1;
      info[i].energy = d.energy;
    }
  }
  return (gn_status)worst;
}

extern "C" float gn_batch_last_ms(gn_batch* b) {
  float ms = 0.0f;
  if (b && b->has_state) cudaEventElapsedTime(&ms, b->ev0, b->ev1);
  return ms;
}

extern "C" gn_status gn_batch_tune(gn_batch* b, const gn_params* p, int max_iters, int* threads_out) {
  using namespace gn;
  if (!b || max_iters < 1) return fail(GN_ERR_ARG, "gn_batch_tune: bad argument");
  // the schedule: CTA size x the size threshold of warp mode (0: every instance a CTA); a
  // threshold that moves no further instance into warp mode than a smaller one is skipped
  const int cand_t[] = {256, 512, 1024};
  const int cand_w[] = {0, 64, 128, 256, 512};
  float best = 1e30f;
  int best_t = b->threads, best_w = b->wmax;
  for (int t : cand_t) {
    int last_small = -1;
    for (int wm : cand_w) {
      b->wmax = wm;
      gn_status st = gn_batch_set_threads(b, t);
      if (st != GN_OK) break;
      const int nsmall = b->count - b->nbig;
      if (nsmall == last_small) continue;
      last_small = nsmall;
      float acc = 0.0f;
      for (int rep = 0; rep < 2; ++rep) {
        st = gn_batch_run(b, nullptr, max_iters, -1.0, p, nullptr, nullptr);
        if (st < 0) return st;
        if (rep) acc += gn_batch_last_ms(b);
      }
      if (acc < best) {
        best = acc;
        best_t = t;
        best_w = wm;
      }
    }
  }
  b->wmax = best_w;
  gn_status st = gn_batch_set_threads(b, best_t);
  if (st != GN_OK) return st;
  if (threads_out) *threads_out = best_t;
  return GN_OK;
}

extern "C" gn_status gn_batch_extract(gn_batch* b, uint8_t* mask, int32_t* counts, double* weights,
                                      int32_t* statuses) {
  using namespace gn;
  if (!b) return fail(GN_ERR_ARG, "gn_batch_extract: NULL handle");
  if (!b->has_state) return fail(GN_ERR_ARG, "gn_batch_extract: no state (run first)");
  if (b->count == 0) return GN_OK;
  k_batch_extract<<<b->count, 256, 0, b->stream>>>(b->count, b->d_vtx_off, b->d_ent_off, b->d_rp, b->d_ci,
                                                    b->d_kind, b->d_x, b->d_w, b->d_mask, b->d_xstatus,
                                                    b->d_xcount, b->d_xweight);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  cudaMemcpyKind k = b->io_mem == GN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (mask) GN_CUDA(cudaMemcpyAsync(mask, b->d_mask, (size_t)b->ntot, k, b->stream));
  if (counts) GN_CUDA(cudaMemcpyAsync(counts, b->d_xcount, sizeof(int32_t) * b->count, k, b->stream));
  if (weights) GN_CUDA(cudaMemcpyAsync(weights, b->d_xweight, sizeof(double) * b->count, k, b->stream));
  std::vector<int32_t> st(b->count);
  GN_CUDA(cudaMemcpyAsync(st.data(), b->d_xstatus, sizeof(int32_t) * b->count, cudaMemcpyDeviceToHost, b->stream));
  GN_CUDA(cudaStreamSynchronize(b->stream));
  if (statuses) {
    if (b->io_mem == GN_DEVICE) GN_CUDA(cudaMemcpy(statuses, st.data(), sizeof(int32_t) * b->count, cudaMemcpyHostToDevice));
    else memcpy(statuses, st.data(), sizeof(int32_t) * b->count);
  }
  int worst = GN_OK;
  for (int s : st) {
    if (s < 0) return fail(GN_ERR_NOT_INDEPENDENT, "gn_batch_extract: an instance's rounded set is not independent");
    worst = std::max(worst, s);
  }
  return (gn_status)worst;
}
