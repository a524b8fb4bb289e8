// gn_iter_common.cuh -- the parts of one WRGN iteration that every gather mode shares:
// the per-vertex update (App. B weighted state, float-pair own state), the stop-test
// partials, the bounded grid barrier and the stop decision.
#pragma once

#include "gn_device.cuh"

namespace gn {

// launch parameters of the persistent kernels
struct IterParams {
  const int32_t* row_ptr;
  const int32_t* col_idx;
  const float* v;       // v_hi
  const float* vlo;     // v_lo
  const float* w;
  const int32_t* part;
  float* y0;            // holds y^{k_start}
  float* y1;
  float* x;             // holds x^{k_start}; receives the final x (internal order)
  float* ylo;           // Own::aux of every row (in and out)
  float* yexp;          // Own::xs of the rows whose state is scaled, else 0 (in and out)
  CheckPartial* partials;
  unsigned* bar;
  int* status;
  DevInfo* info;
  // halo mode (gn_halo.cu): per-CTA blocks of a packed layout, see HaloLayout
  const int64_t* hoff;      // [nblocks + 1] byte offsets of each CTA's block in hblob
  const unsigned char* hblob;
  const float2* gtab;       // gamma_k as float pairs for k < gtab_len (then the last entry)
  int gtab_len;
  int n, nblocks;
  int k_start, k_end;
  int gamma_mode;
  double gamma0, gamma1;
  int ramp;
  int check_every;
  double theta;
  double tol;
  // the stop test without FP64 on the device: gamma (1 - theta) > theta as gamma > thr, thr =
  // theta / (1 - theta) as a float pair; the residual test as r <= tol_f, tol_f the largest
  // float <= tol (exact for an FP32 r), on when res_test
  float thr_hi, thr_lo;
  float tol_f;
  int res_test;
  int heavy;
  int rows_pad;
  int halo_pad;
  long long spin_limit;
  int unreachable;
  int bad_tag;  // test hook (tagged exchange): the first halo wait expects a tag no value carries
  // halo mode: three exchange buffers of inbox_len floats (push: the per-CTA inboxes, of which
  // the barrier and the flags use two; pull: a slot per vertex, for the tagged exchange)
  float* inbox;
  long long inbox_len;
  // neighbour synchronisation (halo mode): iterflag[kFlagStride * b] counts the pushes CTA b
  // has completed in this launch (zeroed before it); nullptr = a grid barrier every iteration
  unsigned* iterflag;
};

static constexpr int kThreads = 1024;
static constexpr float kSafeDiv = 1e-9f;

// per-CTA shared arrays of the owned rows (each row's own state is the triple (yh, yl, x),
// see Own)
struct RowArrays {
  float* sum;   // neighbour sums s_i of this iteration
  float* yh;    // Own::pub
  float* yl;    // Own::aux
  float* x;     // Own::xs
  float* vh;    // v = sqrt(w), float pair
  float* vl;
};

// Safe-division hits are counted per thread in 32 bits (a call runs fewer than 2^31 / nblocks
// iterations and a thread updates a few rows per iteration) and summed in 64 bits per CTA.

// per-thread accumulators of the stop test
struct CheckAcc {
  float rmax = 0.0f;
  unsigned nonbin = 0;
  float l1 = 0.0f, obj = 0.0f, en = 0.0f;
};

// The own state of a row, three words with an exponent range beyond FP32's.  Non-members decay
// geometrically (App. G: by 1 / (gamma sum_{j in N(i) cap M} v_j / v_i) per step), so after a few
// hundred steps many are far below FP32's smallest normal 2^-126.  Whether such a vertex comes
// back later -- its neighbours decaying faster than it does, until x_i / d_i grows -- depends on
// how deep it is, which FP32 would lose by storing 0.  The own state therefore carries its own
// binary exponent; the value neighbours gather stays FP32, since a term below 2^-126 cannot move
// a sum d_i = (B y)_i that is above the 1e-9 of the safe division.
//   xs >= 0: y = pub + aux (float pair), x = xs;
//   xs <  0: x < 2^-64, taken as 0 by the stop test; y = aux * 2^xs (xs a negative multiple of 64,
//            aux the FP32 mantissa); pub = y in FP32 at xs = -64, 0 further down.
// pub is the value the neighbours gather in both cases.
struct Own {
  float pub, aux, xs;
};
__device__ __forceinline__ bool own_scaled(const Own& s) { return s.xs < 0.0f; }
// 2^e for e in {0, -64, -128, ...} as an FP32 value: 1, 2^-64, 2^-128 (subnormal), 0 below
__device__ __forceinline__ float pow2_scale(float e) {
  return e == 0.0f ? 1.0f : (e == -64.0f ? __int_as_float(0x1f800000) : (e == -128.0f ? __int_as_float(0x00200000) : 0.0f));
}
// the x of an own state as an FP32 value (the run's output): x = y / v
__device__ __forceinline__ float own_x(const Own& s, float vh) {
  return own_scaled(s) ? __fdiv_rn(s.aux, vh) * pow2_scale(s.xs) : s.xs;
}
// the own state of a run's start or of a saved state: pub / aux / x as stored, xe the saved
// exponent (0 unless the state was scaled)
__device__ __forceinline__ Own own_load(float pub, float aux, float x, float xe) {
  return xe < 0.0f ? Own{pub, aux, xe} : Own{pub, aux, x};
}

// The update of one row (global id rb + i), arithmetic only:
//   d = y + gamma s = (B y)_i, x' = y / d, y' = v x'  (Def. 3, WRGN, in the weighted state of Sec. 3 / App. B)
//   d <= 1e-9: x' = 1/2 (the safe division of the appendix module)
// The quotient is taken on the mantissa of y (y = m 2^e), so x' = (m / d) 2^e has the range of
// the own state; after the step the mantissa is rescaled by 2^64 when x' drops below 2^-64, or
// when it is back at or above 2^-64 with e < 0.  For rows that never go below 2^-64 this is
// exactly the float-pair update.  A scaled row's x is taken as 0 in the stop test and in the
// objective (it is below 2^-64), and its gathered value is exact at e = -64 and 0 further down
// (below 2^-104 v, nothing next to a sum above the safe-division threshold).  Straight-line
// code (the safe division is a select), so a thread's rows can interleave.
struct RowStep {
  Own next;        // the new own state
  float x;         // x' as an FP32 value (0 for a scaled row)
  float yin;       // y before the step as an FP32 value (the energy term)
  float d;         // (B y)_i, hi part (the energy term)
  bool ok;         // false: the safe division fired
};
__device__ __forceinline__ RowStep update_core(const Own s, const dev::f2 v, float sn, dev::f2 gam) {
  const bool sc = own_scaled(s);
  const float e = fminf(s.xs, 0.0f);
  const float mh = sc ? s.aux : s.pub, ml = sc ? 0.0f : s.aux;  // y = (mh + ml) 2^e
  dev::f2 p = dev::two_prod(gam.hi, sn);
  p.lo = dev::ffma(gam.lo, sn, p.lo);
  dev::f2 d = dev::two_sum(s.pub, p.hi);                         // y in FP32 range: (pub, ml)
  d = dev::fast_two_sum(d.hi, dev::fadd(d.lo, dev::fadd(ml, p.lo)));
  RowStep r;
  r.ok = d.hi > kSafeDiv;
  const dev::f2 q = dev::div_f2(dev::f2{mh, ml}, r.ok ? d : dev::f2{1.0f, 0.0f});
  const dev::f2 xm = r.ok ? q : dev::f2{0.5f, 0.0f};            // x' = xm 2^ex
  const float ex = r.ok ? e : 0.0f;
  dev::f2 ym = dev::mul_f2(v, xm);                                // y' = ym 2^ex
  const bool down = xm.hi < 0x1p-64f && xm.hi > 0.0f;
  const bool neg = ex < 0.0f;
  const bool up = neg && xm.hi >= 1.0f;
  const float f = down ? 0x1p64f : (up ? 0x1p-64f : 1.0f);
  const float en = ex + (down ? -64.0f : (up ? 64.0f : 0.0f));
  ym.hi = dev::fmul(ym.hi, f);
  ym.lo = dev::fmul(ym.lo, f);
  r.x = neg ? 0.0f : xm.hi;
  const bool nsc = en < 0.0f;
  const float sp = en == -64.0f ? 0x1p-64f : 0.0f;
  r.next = Own{nsc ? dev::fmul(ym.hi, sp) : ym.hi, nsc ? ym.hi : ym.lo, nsc ? en : r.x};
  r.yin = s.pub;
  r.d = d.hi;
  return r;
}
// a row's terms of the stop test (FP32 terms, summed as float pairs later): s, v are the state
// and v before the step
__device__ __forceinline__ void check_terms(const RowStep& r, const Own& s, const dev::f2 v, float wi,
                                            float th_lo, float th_hi, CheckAcc& acc) {
  const float dx = fabsf(r.x - (own_scaled(s) ? 0.0f : s.xs));
  acc.rmax = fmaxf(acc.rmax, dx);
  acc.l1 += dx;
  acc.obj = __fmaf_rn(wi, r.x, acc.obj);
  acc.en = __fmaf_rn(r.yin, __fmaf_rn(0.5f, r.d, -v.hi), acc.en);
  acc.nonbin += (r.x > th_lo && r.x < th_hi) ? 1u : 0u;
}
// the update of one row with, at a check, its stop-test terms
__device__ __forceinline__ void update_one(Own& s, const dev::f2 v, float sn, dev::f2 gam, bool check, float wi,
                                           float th_lo, float th_hi, unsigned& hits, CheckAcc& acc) {
  const RowStep r = update_core(s, v, sn, gam);
  hits += r.ok ? 0u : 1u;
  if (check) check_terms(r, s, v, wi, th_lo, th_hi, acc);
  s = r.next;
}

// the update of rows [0, nr) of the CTA with their state in shared memory (and, unless yout is
// null, the new gathered values to global memory)
__device__ __forceinline__ void update_rows(const RowArrays& S, int nr, int rb, const float* __restrict__ w,
                                            float* __restrict__ yout, dev::f2 gam, bool check,
                                            float th_lo, float th_hi, unsigned& hits,
                                            CheckAcc& acc) {
  // rows i and i + blockDim.x together: their arithmetic has no branch between it, so the two
  // dependency chains interleave (a row past the end computes on a fixed point and stores nothing)
  const int step = blockDim.x;
  for (int i = threadIdx.x; i < nr; i += 2 * step) {
    const int i2 = i + step;
    const bool in2 = i2 < nr;
    const Own s1 = {S.yh[i], S.yl[i], S.x[i]};
    const Own s2 = in2 ? Own{S.yh[i2], S.yl[i2], S.x[i2]} : Own{1.0f, 0.0f, 1.0f};
    const dev::f2 v1 = {S.vh[i], S.vl[i]};
    const dev::f2 v2 = in2 ? dev::f2{S.vh[i2], S.vl[i2]} : dev::f2{1.0f, 0.0f};
    const RowStep r1 = update_core(s1, v1, S.sum[i], gam);
    const RowStep r2 = update_core(s2, v2, in2 ? S.sum[i2] : 0.0f, gam);
    if (check) {
      check_terms(r1, s1, v1, w[rb + i], th_lo, th_hi, acc);
      if (in2) check_terms(r2, s2, v2, w[rb + i2], th_lo, th_hi, acc);
    }
    hits += (r1.ok ? 0u : 1u) + (in2 && !r2.ok ? 1u : 0u);
    S.yh[i] = r1.next.pub;
    S.yl[i] = r1.next.aux;
    S.x[i] = r1.next.xs;
    if (yout) yout[rb + i] = r1.next.pub;
    if (in2) {
      S.yh[i2] = r2.next.pub;
      S.yl[i2] = r2.next.aux;
      S.x[i2] = r2.next.xs;
      if (yout) yout[rb + i2] = r2.next.pub;
    }
  }
}

struct TailShared {
  float gh, gl;     // gamma_k of the coming iteration as a float pair
  float rf[32];
  unsigned ru[32];
  float rdh[3][32];
  float rdl[3][32];
  unsigned long long rh[32];
  int decide;
  float last_r;
  unsigned last_n;
};

// block reduction of the stop-test accumulators into this CTA's partial of the check slot
__device__ __forceinline__ void write_check_partial(const IterParams& P, const CheckAcc& a, int slot,
                                                    TailShared& T) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const float rmax = dev::warp_max(a.rmax);
  const unsigned nonbin = dev::warp_sum_u(a.nonbin);
  const dev::f2 l1 = dev::warp_sum_f2(a.l1);
  const dev::f2 obj = dev::warp_sum_f2(a.obj);
  const dev::f2 en = dev::warp_sum_f2(a.en);
  if (lane == 0) {
    T.rf[warp] = rmax;
    T.ru[warp] = nonbin;
    T.rdh[0][warp] = l1.hi;
    T.rdl[0][warp] = l1.lo;
    T.rdh[1][warp] = obj.hi;
    T.rdl[1][warp] = obj.lo;
    T.rdh[2][warp] = en.hi;
    T.rdl[2][warp] = en.lo;
  }
  __syncthreads();
  if (warp == 0) {
    const bool in = lane < nwarps;
    const float r2 = dev::warp_max(in ? T.rf[lane] : 0.0f);
    const unsigned n2 = dev::warp_sum_u(in ? T.ru[lane] : 0u);
    dev::f2 q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
      q[c] = dev::warp_sum_pair(in ? dev::f2{T.rdh[c][lane], T.rdl[c][lane]} : dev::f2{0.0f, 0.0f});
    if (lane == 0) {
      CheckPartial cp;
      cp.rmax = r2;
      cp.nonbin = n2;
      cp.l1h = q[0].hi;
      cp.l1l = q[0].lo;
      cp.objh = q[1].hi;
      cp.objl = q[1].lo;
      cp.enh = q[2].hi;
      cp.enl = q[2].lo;
      P.partials[slot * P.nblocks + blockIdx.x] = cp;
    }
  }
}

// The stop test after every CTA's partial of check slot `slot` is visible: every CTA reduces
// the same partials in the same order, so all take the same decision.  Returns 0 (continue)
// or 1 (stop after this iteration).
// gamma > thr for float pairs (the binarity condition gamma (1 - theta) > theta)
__device__ __forceinline__ bool gamma_above(const IterParams& P, dev::f2 gam) {
  const dev::f2 d = dev::two_sum(gam.hi, -P.thr_hi);
  return dev::fadd(d.hi, dev::fadd(d.lo, dev::fsub(gam.lo, P.thr_lo))) > 0.0f;
}
// float-pair accumulation a += (hi, lo)
__device__ __forceinline__ void add_pair(dev::f2& a, float hi, float lo) {
  const dev::f2 s = dev::two_sum(a.hi, hi);
  a = dev::fast_two_sum(s.hi, dev::fadd(s.lo, dev::fadd(a.lo, lo)));
}

__device__ __forceinline__ int stop_decision(const IterParams& P, int& slot, dev::f2 gam, int k, TailShared& T) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const CheckPartial* cps = P.partials + slot * P.nblocks;
  float fr = 0.0f;
  unsigned fn = 0;
  for (int j = tid; j < P.nblocks; j += blockDim.x) {
    fr = fmaxf(fr, __ldcg(&cps[j].rmax));
    fn += __ldcg(&cps[j].nonbin);
  }
  fr = dev::warp_max(fr);
  fn = dev::warp_sum_u(fn);
  if (lane == 0) {
    T.rf[warp] = fr;
    T.ru[warp] = fn;
  }
  __syncthreads();
  if (tid == 0) {
    float tr = 0.0f;
    unsigned tn = 0;
    for (int j = 0; j < nwarps; ++j) {
      tr = fmaxf(tr, T.rf[j]);
      tn += T.ru[j];
    }
    const bool bin_ok = (tn == 0u) && gamma_above(P, gam);
    const bool res_ok = P.res_test && tr <= P.tol_f;
    const int stop = (bin_ok || res_ok) ? 1 : 0;
    T.decide = stop;
    if (blockIdx.x == 0 && (stop || k + 1 == P.k_end)) {
      // summary of the final step, block 0 only, fixed order, float pairs (one FP64 rounding
      // per quantity at the end)
      dev::f2 a2 = {0.0f, 0.0f}, o2 = {0.0f, 0.0f}, q2 = {0.0f, 0.0f};
      for (int j = 0; j < P.nblocks; ++j) {
        add_pair(a2, __ldcg(&cps[j].l1h), __ldcg(&cps[j].l1l));
        add_pair(o2, __ldcg(&cps[j].objh), __ldcg(&cps[j].objl));
        add_pair(q2, __ldcg(&cps[j].enh), __ldcg(&cps[j].enl));
      }
      P.info->resid_inf = tr;
      P.info->nonbin = tn;
      P.info->resid_l1 = (double)a2.hi + (double)a2.lo;
      P.info->objective = (double)o2.hi + (double)o2.lo;
      P.info->energy = (double)q2.hi + (double)q2.lo;
      P.info->binary = tn == 0u;
      P.info->converged = stop;
    }
  }
  __syncthreads();
  slot ^= 1;
  return T.decide;
}

// The run's summary at its final check (stop, or the last iteration): every CTA writes its full
// partial (slot 0), one more grid barrier, then block 0 reduces the partials in a fixed order
// (float pairs; one FP64 rounding per quantity) and writes the summary.  False if a wait hit
// its limit.
__device__ __forceinline__ bool final_summary(const IterParams& P, unsigned& nbar, const CheckAcc& acc, int stop,
                                              TailShared& T) {
  write_check_partial(P, acc, 0, T);
  ++nbar;
  if (!dev::grid_barrier(P.bar, nbar * (unsigned)P.nblocks + (P.unreachable ? 1u : 0u), P.status, P.spin_limit))
    return false;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    float tr = 0.0f;
    unsigned tn = 0;
    dev::f2 a2 = {0.0f, 0.0f}, o2 = {0.0f, 0.0f}, q2 = {0.0f, 0.0f};
    for (int j = 0; j < P.nblocks; ++j) {
      const CheckPartial* c = P.partials + j;
      tr = fmaxf(tr, __ldcg(&c->rmax));
      tn += __ldcg(&c->nonbin);
      add_pair(a2, __ldcg(&c->l1h), __ldcg(&c->l1l));
      add_pair(o2, __ldcg(&c->objh), __ldcg(&c->objl));
      add_pair(q2, __ldcg(&c->enh), __ldcg(&c->enl));
    }
    P.info->resid_inf = tr;
    P.info->nonbin = tn;
    P.info->resid_l1 = (double)a2.hi + (double)a2.lo;
    P.info->objective = (double)o2.hi + (double)o2.lo;
    P.info->energy = (double)q2.hi + (double)q2.lo;
    P.info->binary = tn == 0u;
    P.info->converged = stop;
  }
  return true;
}

// The stop test fused into the grid barrier (checks in grid-barrier mode).  A CTA brings two
// flags -- one of its rows is non-binary, one of its residuals is above tol -- and its arrival
// on one of three rotating 64-bit check words adds 1 (bits 0..20, arrivals), the first flag
// (bits 21..41) and the second (bits 42..62).  The poll that sees every arrival reads the two
// counts with it, so all CTAs take the same decision with no further global reads: stop when
// no CTA has a non-binary row and gamma (1 - theta) > theta, or when no residual exceeds tol.
// Block 0 clears the previous check's word (every CTA read it before arriving here); that word
// is used again three checks later, after barriers block 0 crosses only after clearing it.
// Returns 0 (continue), 1 (stop after this iteration) or 2 (a wait hit its limit).
__device__ __forceinline__ int check_barrier(const IterParams& P, bool may_fail, bool fail, unsigned& nbar,
                                             int& nchk, dev::f2 gam, int k, const CheckAcc& acc, TailShared& T) {
  __shared__ int s_ok;
  const bool nb_any = __syncthreads_or(acc.nonbin != 0u) != 0;
  const bool rf_any = __syncthreads_or(acc.rmax > P.tol_f) != 0;
  if (may_fail && __syncthreads_or(fail)) return 2;
  unsigned long long* words = reinterpret_cast<unsigned long long*>(P.bar + 2);
  const int w = nchk % 3;
  if (threadIdx.x == 0) {
    constexpr unsigned long long kField = (1ull << 21) - 1ull;
    dev::red_release_add_u64(words + w, 1ull | (nb_any ? 1ull << 21 : 0ull) | (rf_any ? 1ull << 42 : 0ull));
    const unsigned long long need = (unsigned long long)P.nblocks + (P.unreachable ? 1ull : 0ull);
    int ok = 1;
    long long spins = 0;
    unsigned long long v;
    while (((v = dev::ld_acquire_u64(words + w)) & kField) < need) {
      ++spins;
      if ((spins & 255) == 0 && dev::ld_relaxed_int(P.status) != 0) { ok = 0; break; }
      if (spins > P.spin_limit) {
        atomicOr(P.status, DEV_TIMEOUT);
        ok = 0;
        break;
      }
    }
    int stop = 0;
    if (ok) {
      const bool bin_ok = ((v >> 21) & kField) == 0ull && gamma_above(P, gam);
      const bool res_ok = P.res_test && ((v >> 42) & kField) == 0ull;
      stop = (bin_ok || res_ok) ? 1 : 0;
      if (blockIdx.x == 0) dev::st_relaxed_u64(words + (w + 2) % 3, 0ull);
    }
    s_ok = ok;
    T.decide = stop;
  }
  __syncthreads();
  if (!s_ok) return 2;
  ++nchk;
  const int stop = T.decide;
  if (stop || k + 1 == P.k_end) {
    if (!final_summary(P, nbar, acc, stop, T)) return 2;
  }
  return stop;
}

// Grid barrier, then (at a check) the stop test.  `fail` is this thread's record of a wait
// that hit its limit earlier in the iteration; `may_fail` (a constant at the call site) says
// whether the kernel has such waits.  Returns 0 (continue), 1 (stop after this iteration) or 2
// (a wait hit its limit).
__device__ __forceinline__ int barrier_and_stop(const IterParams& P, bool may_fail, bool fail, unsigned& nbar,
                                                int& slot, bool check, dev::f2 gam, int k, TailShared& T) {
  ++nbar;
  const unsigned target = nbar * (unsigned)P.nblocks + (P.unreachable ? 1u : 0u);
  if (!dev::grid_barrier(P.bar, target, P.status, P.spin_limit, may_fail, fail)) return 2;
  if (!check) return 0;
  return stop_decision(P, slot, gam, k, T);
}

// Neighbour synchronisation, end of iteration k (k = k_start - 1: the prologue): once every
// thread's writes of the iteration (its pushed states, the check partial) are done, thread 0
// publishes the CTA's count of completed pushes, k + 2 - k_start, with a release store.
// Between checks nothing more: the next iteration's readers wait for the flags they need
// (wait_flags_warp).  At a check the stop test needs every CTA's partial, so warp 0 waits for
// all flags first.  `fail` is this thread's record of a wait that hit its limit earlier in the
// iteration.  Returns 0, 1 or 2 like barrier_and_stop.
__device__ __forceinline__ int publish_and_stop(const IterParams& P, bool fail, int& slot, bool check,
                                                dev::f2 gam, int k, TailShared& T) {
  __shared__ int s_ok;
  if (__syncthreads_or(fail)) return 2;
  const unsigned done = (unsigned)(k + 2 - P.k_start);
  if (threadIdx.x == 0) dev::st_release(P.iterflag + dev::kFlagStride * blockIdx.x, done);
  if (!check) return 0;
  if (threadIdx.x < 32) {
    const bool ok = dev::wait_flags_warp(P.iterflag, nullptr, P.nblocks, done + (P.unreachable ? 1u : 0u),
                                         P.status, P.spin_limit);
    if (threadIdx.x == 0) s_ok = ok;
  }
  __syncthreads();
  if (!s_ok) return 2;
  return stop_decision(P, slot, gam, k, T);
}

// gamma_k (Sec. 6) for iteration k from the per-run table (float pair; FP64 value = hi + lo),
// read by thread 0 and broadcast through shared memory.  The load for iteration k + 1 is
// issued at the start of iteration k (gamma_fetch) and stored after the update (gamma_store),
// so its latency hides behind the iteration.
__device__ __forceinline__ float2 gamma_fetch(const IterParams& P, int k) {
  return threadIdx.x == 0 ? P.gtab[k < P.gtab_len ? k : P.gtab_len - 1] : make_float2(0.0f, 0.0f);
}
__device__ __forceinline__ void gamma_store(float2 g, TailShared& T) {
  if (threadIdx.x == 0) {
    T.gh = g.x;
    T.gl = g.y;
  }
}
__device__ __forceinline__ void set_gamma(const IterParams& P, int k, TailShared& T) {
  gamma_store(gamma_fetch(P, k), T);
}

// end of a run: own x, the second word of each own state and its exponent back to global memory
// (the gathered values are already there), safe-division count,
// iteration count and the parity of the buffer holding the final weighted state
__device__ __forceinline__ void finish_run(const IterParams& P, const RowArrays& S, int rb, int nr,
                                           unsigned long long hits, int k, int parity, TailShared& T) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  for (int i = tid; i < nr; i += blockDim.x) {
    const Own s = {S.yh[i], S.yl[i], S.x[i]};
    P.x[rb + i] = own_x(s, S.vh[i]);
    P.ylo[rb + i] = s.aux;
    P.yexp[rb + i] = own_scaled(s) ? s.xs : 0.0f;
  }
  unsigned long long h = dev::warp_sum_ull(hits);
  if (lane == 0) T.rh[warp] = h;
  __syncthreads();
  if (tid == 0) {
    unsigned long long t = 0;
    for (int j = 0; j < nwarps; ++j) t += T.rh[j];
    if (t) atomicAdd(&P.info->hits, t);
    if (blockIdx.x == 0) {
      P.info->iters = k - P.k_start;
      P.info->final_parity = parity;
    }
  }
}

}  // namespace gn
