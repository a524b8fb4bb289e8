// gn_device.cuh -- what the library's kernels share: the device status word, the per-CTA
// stop-test partials, the run summary left on the device, and the device helpers (ordered
// loads and reductions, bounded waits and barriers, float-pair arithmetic).  Device code only:
// the host side (the handle, error plumbing, host threads) is in gn_internal.cuh.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gn.h"

namespace gn {

// device-side status word (written by kernels, read once by the host)
enum DevStatus : int {
  DEV_OK = 0,
  DEV_NOT_NORMALIZABLE = 1,
  DEV_TIMEOUT = 2,
  DEV_BAD_CSR = 4,
  DEV_NOT_SIMPLE = 8,
  DEV_BAD_WEIGHT = 16,
};

// per-CTA partial of a stop-test check (double-buffered by check parity).  The sums are float
// pairs (hi + lo): FP64 arithmetic is slow on this GPU and stays off the iteration path.
struct alignas(32) CheckPartial {
  float rmax;           // max |x' - x|
  unsigned nonbin;      // count of theta < x' < 1 - theta
  float l1h, l1l;       // sum |x' - x|
  float objh, objl;     // sum w x'
  float enh, enl;       // sum y (d/2 - v)  (E~ of the state entering the step)
};

// summary the iteration kernels leave on the device (one D2H copy per run)
struct DevInfo {
  int iters;
  int converged;
  int binary;
  int final_parity;     // d_y[final_parity] holds the final weighted state
  float resid_inf;
  unsigned nonbin;
  double resid_l1;
  double objective;
  double energy;
  unsigned long long hits;
  int status;
  int pad;
};

}  // namespace gn

// ------------------------------------------------------------------------------------------
// device helpers

namespace gn {
namespace dev {

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed_int(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() {
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
}
__device__ __forceinline__ void st_relaxed_u32(unsigned* p, unsigned v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier for a cooperative launch (every CTA co-resident).  The counter only
// grows: the e-th barrier of the launch waits for nblocks * (e + 1) arrivals.  The wait is
// bounded: after `spin_limit` polls (or when another CTA has already reported a failure)
// the CTA records DEV_TIMEOUT and returns false, so the kernel can wind down instead of
// hanging.  The arrival is a release reduction (every write of the CTA before the barrier,
// made visible to thread 0 by the bar.sync, is ordered before it); the polls are acquire
// loads, so the one that sees the full count orders every later read (measured on GB300 with
// 152 CTAs: 1.27 us per barrier, against 1.42 us with relaxed polls and a trailing fence).
__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned target, int* status,
                                             long long spin_limit, bool may_fail = false, bool fail = false) {
  __shared__ int s_ok;
  // `fail`: a thread's record of a wait that hit its limit earlier; the CTA then stops here.
  // `may_fail` is a constant at the call site: without such waits a plain bar.sync does.
  if (may_fail) {
    if (__syncthreads_or(fail)) return false;
  } else {
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    red_release_add(counter, 1u);
    int ok = 1;
    long long spins = 0;
    while (ld_acquire(counter) < target) {
      ++spins;
      if ((spins & 255) == 0 && ld_relaxed_int(status) != 0) { ok = 0; break; }
      if (spins > spin_limit) {
        atomicOr(status, DEV_TIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Per-CTA flags sit kFlagStride words apart (a cache line each), so the CTAs polling one flag
// do not contend with those polling another.
static constexpr int kFlagStride = 32;

// One warp waits until flag ids[j] >= target for j < count (ids == nullptr: flag j), flag i
// being flags[kFlagStride * i].
// Relaxed polls (all of a lane's loads in flight together), then an acquire fence in every
// lane, so the releases that set the flags are ordered before the warp's later reads; a
// bar.sync after it extends that to the CTA.  Bounded like grid_barrier; warp-uniform result.
__device__ __forceinline__ bool wait_flags_warp(const unsigned* flags, const int* ids, int count,
                                                unsigned target, int* status, long long spin_limit) {
  const int lane = threadIdx.x & 31;
  long long spins = 0;
  for (;;) {
    bool ok = true;
    for (int j = lane; j < count; j += 32) ok &= ld_relaxed(flags + kFlagStride * (ids ? ids[j] : j)) >= target;
    if (__all_sync(0xffffffffu, ok)) break;
    ++spins;
    if ((spins & 255) == 0) {
      const int bad = lane == 0 ? ld_relaxed_int(status) : 0;
      if (__shfl_sync(0xffffffffu, bad, 0) != 0) return false;
    }
    if (spins > spin_limit) {
      if (lane == 0) atomicOr(status, DEV_TIMEOUT);
      return false;
    }
  }
  fence_acq_rel();
  return true;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ unsigned warp_sum_u(unsigned v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_ull(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- float-pair ("double-float") arithmetic on the FP32 pipes.  A value is hi + lo with
// |lo| <= ulp(hi)/2.  Every operation is explicit round-to-nearest PTX, so the compiler cannot
// contract or reorder the error-free transforms.  Subnormal values are kept (FP32 add, mul
// and fma handle them at full rate); the quotient uses an approximate reciprocal plus a
// correction instead of the IEEE division sequence, whose slow path subnormals would take.
struct f2 {
  float hi, lo;
};
__device__ __forceinline__ float fadd(float a, float b) {
  float r;
  asm("add.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float fsub(float a, float b) {
  float r;
  asm("sub.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float fmul(float a, float b) {
  float r;
  asm("mul.rn.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float ffma(float a, float b, float c) {
  float r;
  asm("fma.rn.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float frcp_approx(float a) {
  float r;
  asm("rcp.approx.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ f2 two_sum(float a, float b) {
  float s = fadd(a, b);
  float bb = fsub(s, a);
  float e = fadd(fsub(a, fsub(s, bb)), fsub(b, bb));
  return {s, e};
}
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {  // requires |a| >= |b| or a == 0
  float s = fadd(a, b);
  return {s, fsub(b, fsub(s, a))};
}
__device__ __forceinline__ f2 two_prod(float a, float b) {
  float p = fmul(a, b);
  return {p, ffma(a, b, -p)};
}
// (a_hi + a_lo) * (b_hi + b_lo), normalised
__device__ __forceinline__ f2 mul_f2(f2 a, f2 b) {
  f2 p = two_prod(a.hi, b.hi);
  float c = ffma(a.hi, b.lo, fmul(a.lo, b.hi));
  return fast_two_sum(p.hi, fadd(p.lo, c));
}
// a / b for float pairs, b.hi a normal number: an approximate reciprocal, a quotient, its exact
// residual a - q1 b, and one correction (relative error about 2^-44)
__device__ __forceinline__ f2 div_f2(f2 a, f2 b) {
  const float r0 = frcp_approx(b.hi);
  const float q1 = fmul(a.hi, r0);
  const f2 t = two_prod(q1, b.hi);
  const float rem = fadd(fsub(fsub(a.hi, t.hi), t.lo), fsub(a.lo, fmul(q1, b.lo)));
  const float q2 = fmul(rem, r0);
  return fast_two_sum(q1, q2);
}
__device__ __forceinline__ f2 split_f64(double v) {
  float hi = __double2float_rn(v);
  return {hi, __double2float_rn(v - (double)hi)};
}
// warp sum of float pairs (compensated), for FP64-grade totals on the FP32 pipes
__device__ __forceinline__ f2 warp_sum_pair(f2 a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float oh = __shfl_xor_sync(0xffffffffu, a.hi, o);
    const float ol = __shfl_xor_sync(0xffffffffu, a.lo, o);
    f2 s = two_sum(a.hi, oh);
    a = fast_two_sum(s.hi, fadd(s.lo, fadd(a.lo, ol)));
  }
  return a;
}
__device__ __forceinline__ f2 warp_sum_f2(float v) { return warp_sum_pair(f2{v, 0.0f}); }

// gamma_k of Sec. 6 / the appendix module, in FP64 (then rounded once to FP32 by callers)
__device__ __forceinline__ double gamma_at(int mode, double g0, double g1, int T, int k) {
  if (mode == GN_GAMMA_FIXED || T <= 1) return g1;
  int kk = k < T - 1 ? k : T - 1;
  double t = __ddiv_rn((double)kk, (double)(T - 1));
  return __dadd_rn(__dmul_rn(t, g1), __dmul_rn(__dsub_rn(1.0, t), g0));  // no contraction
}

}  // namespace dev
}  // namespace gn
