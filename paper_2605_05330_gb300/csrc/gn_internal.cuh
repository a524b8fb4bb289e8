// gn_internal.cuh -- shared host-side internals of libgn.so (handle layout, error plumbing,
// host threads); the kernels' shared device code is in gn_device.cuh.  Not part of the public
// ABI (include/gn.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#ifdef __linux__
#include <sched.h>
#endif

#include <algorithm>
#include <atomic>
#include <functional>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "gn.h"
#include "gn_device.cuh"

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
  float* d_ylo = nullptr;       // second words of the vertices' own states after a run (gn::Own::aux)
  float* d_yexp = nullptr;      // their exponents (gn::Own::xs of a scaled state, else 0)
  int state_parity = 0;         // d_y[state_parity] holds the high parts of that state
  float* d_io = nullptr;        // staging for x0 / outputs (caller order)
  float* d_tmp = nullptr;       // internal-order scratch state
  double* d_bsum = nullptr;     // per-CTA FP64 partial sums of the small reductions
  gn::CheckPartial* d_partials = nullptr;  // [2][nblocks]
  unsigned* d_bar = nullptr;   // [8]: grid-barrier counter, then three 64-bit check words (bytes 8..31)
  unsigned* d_iterflag = nullptr;  // [kFlagStride * nblocks] per-CTA push counts (halo mode)
  float* d_inbox = nullptr;        // [3][inbox_len] halo exchange buffers (halo mode): push, the
                                   // inboxes; pull, a slot per vertex for the tagged exchange
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
gn_status rcm_reorder_device(gn_graph* g, std::vector<int32_t>& rp, std::unique_ptr<int32_t[]>& ci_new,
                             bool* done);
// implemented in gn_graph.cu
gn_status upload_or_alias(gn_graph* g, const void* src, size_t bytes, const void** dev_ptr);
gn_status copy_out(gn_graph* g, void* dst, const void* dev_src, size_t bytes);

// Host-side preparation work over [0, n) split into contiguous blocks, one per host thread
// (at most the hardware's count, and one per `grain` items): body(lo, hi, thread).  The
// blocks are fixed by n and the thread count only, and every caller writes disjoint outputs,
// so results do not depend on scheduling.  The blocks run on a pool of worker threads started
// once per process (run_parts, gn_graph.cu): a block costs a wake-up, not a thread start.
// The thread count is the CPUs this process may run on (its affinity mask, which a container's
// CPU set limits), else the hardware's count; at most 64.
inline int host_threads() {
  static const int count = [] {
    unsigned h = std::thread::hardware_concurrency();
#ifdef __linux__
    cpu_set_t set;
    CPU_ZERO(&set);
    if (sched_getaffinity(0, sizeof set, &set) == 0 && CPU_COUNT(&set) > 0) h = (unsigned)CPU_COUNT(&set);
#endif
    return (int)std::max(1u, std::min(h == 0 ? 1u : h, 64u));
  }();
  return count;
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
