// gn_internal.cuh -- shared internals of libgn.so (handle layout, error plumbing, device
// helpers).  Not part of the public ABI (include/gn.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>
#include <functional>
#include <string>
#include <thread>
#include <vector>

#include "gn.h"

namespace gn {

// ------------------------------------------------------------------------------------------
// error plumbing

void set_error(const std::string& msg);
gn_status fail(gn_status st, const std::string& msg);
gn_status cuda_fail(cudaError_t e, const char* what);

// every kernel launch of the library goes through GN_LAUNCHED() right after the <<<>>>
void count_launch(int k = 1);
#define GN_LAUNCHED() ::gn::count_launch()

#define GN_CUDA(call)                                          \
  do {                                                         \
    cudaError_t e__ = (call);                                  \
    if (e__ != cudaSuccess) return ::gn::cuda_fail(e__, #call); \
  } while (0)

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

struct RecordState;   // gn_adjoint.cu

}  // namespace gn

// ------------------------------------------------------------------------------------------
// the handle

struct gn_graph {
  int device = 0;
  int num_sms = 0;
  int io_mem = GN_HOST;
  cudaStream_t stream = nullptr;

  int32_t n = 0;
  int64_t nnz = 0;
  int reorder = GN_REORDER_NONE;
  int reorder_where = 0;         // GN_ORDER_FROM_HOST / _DEVICE, 0 without reordering

  // graph (internal vertex order)
  int32_t* d_row_ptr = nullptr;
  int32_t* d_col_idx = nullptr;
  float* d_w = nullptr;
  float* d_v = nullptr;         // v = sqrt(w) rounded to FP32 (high part)
  float* d_vlo = nullptr;       // sqrt(w) - v_hi (low part of the float pair)
  int32_t* d_perm = nullptr;    // perm[internal] = caller id (nullptr if no reorder)
  int32_t* d_iperm = nullptr;   // iperm[caller] = internal id

  // persistent-kernel partition: CTA b owns internal rows [part[b], part[b+1])
  int nblocks = 0;
  int32_t* d_part = nullptr;
  int max_rows = 0;             // max rows of one CTA
  int64_t max_ents = 0;         // max CSR entries of one CTA
  int group = 4;                // lanes per light row
  int heavy = 128;              // rows with more entries go warp-per-row
  bool csr_in_smem = false;
  int mode = 0;                 // gather mode of the persistent kernel (gn_iterate.cu)
  int gather = 0;               // requested GN_GATHER_* at create, then the one in use
  int halo_pad = 0;             // padded length of the longest per-CTA halo list
  int rows_pad_halo = 0;        // padded rows per CTA of the halo layout
  void* d_gtab = nullptr;       // per-run gamma_k table (float pairs)
  int gtab_cap = 0;
  int64_t* d_hoff = nullptr;    // [nblocks + 1] byte offsets of the per-CTA halo blocks
  unsigned char* d_hblob = nullptr;  // packed per-CTA halo blocks (gn_halo.cu)
  size_t smem_bytes = 0;
  int threads = 1024;

  // state and scratch (device)
  float* d_y[2] = {nullptr, nullptr};
  float* d_x = nullptr;         // last returned state (internal order, clamped)
  float* d_ylo = nullptr;       // low parts of the vertices' own weighted states after a run
  int state_parity = 0;         // d_y[state_parity] holds the high parts of that state
  float* d_io = nullptr;        // staging for x0 / outputs (caller order)
  float* d_tmp = nullptr;       // internal-order scratch state
  double* d_bsum = nullptr;     // per-CTA FP64 partial sums of the small reductions
  gn::CheckPartial* d_partials = nullptr;  // [2][nblocks]
  unsigned* d_bar = nullptr;   // [8]: grid-barrier counter, then three 64-bit check words (bytes 8..31)
  unsigned* d_iterflag = nullptr;  // [kFlagStride * nblocks] per-CTA push counts (halo mode)
  float* d_inbox = nullptr;        // [2][inbox_len] halo inboxes (halo mode, push exchange)
  bool halo_push = false;          // halo mode: push exchange (else pull)
  int64_t inbox_len = 0;
  gn::DevInfo* d_info = nullptr;
  gn::DevInfo* h_info = nullptr;           // pinned
  int* d_flags = nullptr;
  int* h_flags = nullptr;                  // pinned
  double* d_red = nullptr;                 // small FP64 scratch for reductions
  double* h_red = nullptr;                 // pinned
  // gn_create's fixed-size buffers live in one device allocation and one pinned host allocation;
  // the pointers into them are freed with them, not one by one
  unsigned char* d_arena = nullptr;
  size_t arena_bytes = 0;
  unsigned char* h_arena = nullptr;
  uint8_t* d_mask = nullptr;    // rounded set, internal order
  uint8_t* d_mask_c = nullptr;  // rounded set, caller order
  int* d_bcount = nullptr;      // per-CTA member counts / offsets (extraction)
  double* d_bws = nullptr;      // per-CTA W(S) partials (extraction)
  int32_t* d_members = nullptr;
  bool has_state = false;

  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  gn::RecordState* rec = nullptr;          // checkpoints for gn_backward
  gn_batch* cta = nullptr;                 // GN_KERNEL_CTA: a one-instance batch over this CSR
  int64_t* d_cta_off = nullptr;            // its offsets (vertices, entries)
  bool state_cta = false;                  // the last run was a CTA-kernel run (not resumable)
};

namespace gn {

// implemented in gn_iterate.cu
gn_status run_iterations(gn_graph* g, int k_start, int k_end, double tol, const gn_params& p,
                         int parity0, DevInfo* out, float* ms, int* kernel_used);
gn_status init_state(gn_graph* g, const float* x0_dev_caller_order);
double host_gamma(const gn_params& p, int k);
// implemented in gn_extract.cu
gn_status state_stats(gn_graph* g, const float* x_int, double theta, double* obj, unsigned* nonbin);
gn_status to_internal(gn_graph* g, const float* x_caller, const float** x_int);
// implemented in gn_reorder.cu
gn_status rcm_order_device(gn_graph* g, const std::vector<int32_t>& rp, std::vector<int32_t>& perm,
                           bool* done);
// implemented in gn_graph.cu
gn_status upload_or_alias(gn_graph* g, const void* src, size_t bytes, const void** dev_ptr);
gn_status copy_out(gn_graph* g, void* dst, const void* dev_src, size_t bytes);

// Host-side preparation work over [0, n) split into contiguous blocks, one per host thread
// (at most the hardware's count, and one per `grain` items): body(lo, hi, thread).  The
// blocks are fixed by n and the thread count only, and every caller writes disjoint outputs,
// so results do not depend on scheduling.  The blocks run on a pool of worker threads started
// once per process (run_parts, gn_graph.cu): a block costs a wake-up, not a thread start.
inline int host_threads() {
  const unsigned h = std::thread::hardware_concurrency();
  return (int)std::max(1u, std::min(h == 0 ? 1u : h, 64u));
}
// runs f(0) .. f(parts - 1), parts <= host_threads(), concurrently; returns when all are done
void run_parts(int parts, const std::function<void(int)>& f);
template <class F>
void parallel_for(int n, int grain, F&& body) {
  const int nt = std::max(1, std::min(host_threads(), (n + std::max(grain, 1) - 1) / std::max(grain, 1)));
  if (nt <= 1) {
    if (n > 0) body(0, n, 0);
    return;
  }
  run_parts(nt, [&body, n, nt](int t) {
    body((int)((int64_t)n * t / nt), (int)((int64_t)n * (t + 1) / nt), t);
  });
}
// Items [0, n) of uneven cost, handed to the host threads one at a time: body(item, thread).
// Every item's output is its own; `thread` (< host_threads()) only selects scratch space.
template <class F>
void parallel_items(int n, F&& body) {
  const int nt = std::max(1, std::min(host_threads(), n));
  if (nt <= 1) {
    for (int i = 0; i < n; ++i) body(i, 0);
    return;
  }
  std::atomic<int> next{0};
  run_parts(nt, [&body, &next, n](int t) {
    for (int i = next.fetch_add(1, std::memory_order_relaxed); i < n; i = next.fetch_add(1, std::memory_order_relaxed))
      body(i, t);
  });
}

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
