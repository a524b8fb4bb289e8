// gn_graph.cu -- a1 of the path: gn_create / gn_destroy.  Uploads the CSR and weights,
// validates them on the device (Sec. 2: simple undirected graph; Def. WRGN: w > 0),
// computes v = sqrt(w), optionally reorders the vertices (RCM or by degree) for gather
// locality, and partitions the rows across the persistent kernel's CTAs.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <vector>

#include <unistd.h>

#include "gn_internal.cuh"

namespace gn {

static thread_local std::string t_last_error;
static std::atomic<long long> g_launches{0};

void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

void set_error(const std::string& msg) { t_last_error = msg; }

gn_status fail(gn_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

gn_status cuda_fail(cudaError_t e, const char* what) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  return fail(GN_ERR_CUDA, buf);
}

// ------------------------------------------------------------------------------------------
// validation kernels

// rows: entries in range, strictly increasing (sorted, no duplicates), no self-loop
__global__ void k_check_rows(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
                             int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = 0;
  int b = rp[i], e = rp[i + 1];
  int prev = -1;
  for (int k = b; k < e; ++k) {
    int j = ci[k];
    if (j < 0 || j >= n) { f |= DEV_BAD_CSR; break; }
    if (j == i || j <= prev) f |= DEV_NOT_SIMPLE;
    prev = j;
  }
  if (f) atomicOr(flags, f);
}

// symmetry: for every entry (i, j), i appears in row j (binary search; rows are sorted)
__global__ void k_check_symmetry(int n, int64_t nnz, const int32_t* __restrict__ rp,
                                 const int32_t* __restrict__ ci, int* flags) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnz) return;
  // row of entry e: the last i with rp[i] <= e
  int lo = 0, hi = n;  // invariant: rp[lo] <= e < rp[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if ((int64_t)rp[mid] <= e) lo = mid; else hi = mid;
  }
  int i = lo, j = ci[e];
  int a = rp[j], b = rp[j + 1] - 1;
  bool found = false;
  while (a <= b) {
    int m = (a + b) >> 1;
    int c = ci[m];
    if (c == i) { found = true; break; }
    if (c < i) a = m + 1; else b = m - 1;
  }
  if (!found) atomicOr(flags, DEV_NOT_SIMPLE);
}

// weights: finite and positive; v = sqrt(w) (Def. WRGN), kept as a float pair v_hi + v_lo
// (an FP64 square root split once), so that the map's weight ratios carry no FP32 bias
__global__ void k_weights(int n, const float* __restrict__ w, float* __restrict__ v,
                          float* __restrict__ vlo, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float wi = w[i];
  if (!(wi > 0.0f) || !isfinite(wi)) {
    atomicOr(flags, DEV_BAD_WEIGHT);
    v[i] = 1.0f;
    vlo[i] = 0.0f;
    return;
  }
  dev::f2 p = dev::split_f64(sqrt((double)wi));
  v[i] = p.hi;
  vlo[i] = p.lo;
}

// permuted weights: new vertex r is old vertex perm[r]
__global__ void k_permute_w(int n, const int32_t* __restrict__ perm, const float* __restrict__ w_old,
                            float* __restrict__ w_new) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) w_new[r] = w_old[perm[r]];
}

static unsigned grid_for(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ------------------------------------------------------------------------------------------
// host helpers

gn_status upload_or_alias(gn_graph* g, const void* src, size_t bytes, const void** dev_ptr) {
  if (g->io_mem == GN_DEVICE) {
    *dev_ptr = src;
    return GN_OK;
  }
  GN_CUDA(cudaMemcpyAsync(g->d_io, src, bytes, cudaMemcpyHostToDevice, g->stream));
  *dev_ptr = g->d_io;
  return GN_OK;
}

gn_status copy_out(gn_graph* g, void* dst, const void* dev_src, size_t bytes) {
  if (bytes == 0) return GN_OK;
  GN_CUDA(cudaMemcpyAsync(dst, dev_src, bytes,
                          g->io_mem == GN_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                          g->stream));
  return GN_OK;
}

// ---- the host worker pool behind parallel_for
//
// Workers start on the first multi-block job and stay, parked on a condition variable, for the
// life of the process (a forked child starts its own set).  Jobs run one at a time; a job posted
// from inside a job runs its blocks inline.
namespace {
struct HostPool {
  std::mutex mu;
  std::condition_variable go, done;
  const std::function<void(int)>* job = nullptr;
  unsigned long long gen = 0;
  int parts = 0;
  int pending = 0;   // workers yet to finish the current generation
  int workers = 0;
  pid_t pid = 0;
};
std::mutex g_pool_job;           // one job at a time
HostPool* g_pool = nullptr;      // never freed: its detached workers outlive every handle
thread_local bool t_pool_worker = false;

void pool_worker(HostPool* P, int id) {
  t_pool_worker = true;
  unsigned long long seen = 0;
  std::unique_lock<std::mutex> lk(P->mu);
  for (;;) {
    P->go.wait(lk, [&] { return P->gen != seen; });
    seen = P->gen;
    if (id < P->parts) {
      const std::function<void(int)>* f = P->job;
      lk.unlock();
      (*f)(id);
      lk.lock();
    }
    if (--P->pending == 0) P->done.notify_all();
  }
}
}  // namespace

void run_parts(int parts, const std::function<void(int)>& f) {
  if (parts <= 1 || t_pool_worker) {
    for (int t = 0; t < parts; ++t) f(t);
    return;
  }
  std::lock_guard<std::mutex> job_lock(g_pool_job);
  if (!g_pool || g_pool->pid != getpid()) {
    HostPool* P = new HostPool();
    P->pid = getpid();
    P->workers = host_threads() - 1;
    for (int i = 1; i <= P->workers; ++i) std::thread(pool_worker, P, i).detach();
    g_pool = P;
  }
  HostPool* P = g_pool;
  if (parts > P->workers + 1) {  // not reached through parallel_for
    for (int t = 0; t < parts; ++t) f(t);
    return;
  }
  {
    std::lock_guard<std::mutex> lk(P->mu);
    P->job = &f;
    P->parts = parts;
    P->pending = P->workers;
    ++P->gen;
  }
  P->go.notify_all();
  t_pool_worker = true;  // a job posted from block 0 runs inline too
  f(0);
  t_pool_worker = false;
  std::unique_lock<std::mutex> lk(P->mu);
  P->done.wait(lk, [&] { return P->pending == 0; });
  P->job = nullptr;
}

// Reverse Cuthill-McKee over every component (BFS from a minimum-degree vertex, neighbours
// visited in increasing degree, ties in the order met), reversed, on the host: the order the
// device search (gn_reorder.cu) reproduces, used for graphs outside its scope.  perm[new] = old.
// The vertices are bucketed by degree (a stable counting sort); each BFS step places its new
// neighbours by a stable insertion sort on degree.  key[v] holds the degree with the sign bit
// set once v is placed, so each neighbour costs one random access (the traversal is bound by
// those on graphs with random labels).
static void rcm_order(int n, const std::vector<int32_t>& rp, const int32_t* ci, std::vector<int32_t>& perm) {
  perm.clear();
  perm.reserve(n);
  std::vector<int32_t> key(n);
  int dmax = 0;
  for (int i = 0; i < n; ++i) {
    key[i] = rp[i + 1] - rp[i];
    dmax = std::max(dmax, key[i]);
  }
  std::vector<int32_t> start(dmax + 2, 0), byDeg(n);
  for (int i = 0; i < n; ++i) ++start[key[i] + 1];
  for (int d = 0; d <= dmax; ++d) start[d + 1] += start[d];
  for (int i = 0; i < n; ++i) byDeg[start[key[i]]++] = i;
  constexpr int32_t kPlaced = INT32_MIN;
  for (int s : byDeg) {
    if (key[s] < 0) continue;
    size_t head = perm.size();
    perm.push_back(s);
    key[s] |= kPlaced;
    while (head < perm.size()) {
      const int u = perm[head++];
      const size_t first = perm.size();
      for (int k = rp[u]; k < rp[u + 1]; ++k) {
        const int v = ci[k];
        const int32_t kv = key[v];
        if (kv < 0) continue;
        key[v] = kv | kPlaced;
        size_t pos = perm.size();
        perm.push_back(v);
        while (pos > first && (key[perm[pos - 1]] & INT32_MAX) > kv) {
          perm[pos] = perm[pos - 1];
          --pos;
        }
        perm[pos] = v;
      }
    }
  }
  std::reverse(perm.begin(), perm.end());
}

}  // namespace gn

// ------------------------------------------------------------------------------------------
// public ABI

extern "C" void gn_default_params(gn_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->gamma_mode = GN_GAMMA_PURSUIT;
  p->gamma0 = 0.9;
  p->gamma1 = 1.5;
  p->ramp_iters = 1000;
  p->check_every = 10;
  p->theta_bin = 1e-4;
  p->kernel = GN_KERNEL_AUTO;
  p->record = 0;
  p->spin_limit = 0;
  p->debug_unreachable_barrier = 0;
  p->resume = 0;
}

extern "C" int64_t gn_kernel_launches(void) { return gn::g_launches.load(); }

extern "C" const char* gn_last_error(void) { return gn::t_last_error.c_str(); }

extern "C" int32_t gn_num_vertices(const gn_graph* g) { return g ? g->n : 0; }
extern "C" int64_t gn_num_entries(const gn_graph* g) { return g ? g->nnz : 0; }

extern "C" int gn_vertex_order_source(const gn_graph* g) { return g ? g->reorder_where : 0; }

extern "C" gn_status gn_vertex_order(const gn_graph* g, int32_t* order) {
  if (!g || (!order && g->n > 0)) return gn::fail(GN_ERR_ARG, "gn_vertex_order: bad argument");
  if (g->n == 0) return GN_OK;
  if (!g->d_perm) {
    for (int32_t i = 0; i < g->n; ++i) order[i] = i;
    return GN_OK;
  }
  GN_CUDA(cudaMemcpyAsync(order, g->d_perm, sizeof(int32_t) * g->n, cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  return GN_OK;
}

extern "C" gn_status gn_set_io(gn_graph* g, int mem) {
  if (!g || (mem != GN_HOST && mem != GN_DEVICE)) return gn::fail(GN_ERR_ARG, "gn_set_io: bad argument");
  g->io_mem = mem;
  return GN_OK;
}

void gn_free_record(gn_graph* g);  // gn_adjoint.cu

namespace gn {
// finite and positive, nothing else: the flag only
__global__ void k_check_weights(int n, const float* __restrict__ w, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (!(w[i] > 0.0f) || !isfinite(w[i]))) atomicOr(flags, DEV_BAD_WEIGHT);
}
}  // namespace gn

extern "C" gn_status gn_set_weights(gn_graph* g, const float* w) {
  using namespace gn;
  if (!g || (g->n > 0 && !w)) return fail(GN_ERR_ARG, "gn_set_weights: bad argument");
  const int n = g->n;
  if (n == 0) return GN_OK;
  GN_CUDA(cudaSetDevice(g->device));
  const float* w_dev = nullptr;  // caller order
  gn_status st = upload_or_alias(g, w, sizeof(float) * n, (const void**)&w_dev);
  if (st != GN_OK) return st;
  // validate first, so that a rejected vector leaves the handle's weights as they were
  GN_CUDA(cudaMemsetAsync(g->d_flags, 0, sizeof(int) * 8, g->stream));
  k_check_weights<<<grid_for(n, 256), 256, 0, g->stream>>>(n, w_dev, g->d_flags);
  GN_LAUNCHED();
  GN_CUDA(cudaMemcpyAsync(g->h_flags, g->d_flags, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (g->h_flags[0] & DEV_BAD_WEIGHT) return fail(GN_ERR_WEIGHT, "gn_set_weights: weight <= 0 or not finite");
  if (g->d_perm) {
    k_permute_w<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_perm, w_dev, g->d_w);
    GN_LAUNCHED();
  } else {
    GN_CUDA(cudaMemcpyAsync(g->d_w, w_dev, sizeof(float) * n, cudaMemcpyDeviceToDevice, g->stream));
  }
  k_weights<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_w, g->d_v, g->d_vlo, g->d_flags);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  // what depended on the old weights: the recorded forward, a state to resume from, and the
  // one-instance batch of the CTA kernel (built again on its next use)
  gn_free_record(g);
  if (g->cta) {
    gn_batch_destroy(g->cta);
    g->cta = nullptr;
  }
  g->has_state = false;
  GN_CUDA(cudaStreamSynchronize(g->stream));
  return GN_OK;
}

extern "C" void gn_destroy(gn_graph* g) {
  if (!g) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(g->device);
  if (g->stream) cudaStreamSynchronize(g->stream);
  gn_free_record(g);
  if (g->cta) gn_batch_destroy(g->cta);
  void* dptrs[] = {g->d_row_ptr, g->d_col_idx, g->d_w, g->d_v, g->d_vlo, g->d_ylo, g->d_yexp, g->d_perm, g->d_iperm, g->d_part,
                   g->d_y[0], g->d_y[1], g->d_x, g->d_tmp, g->d_bsum, g->d_io, g->d_partials, g->d_bar, g->d_iterflag, g->d_inbox, g->d_info,
                   g->d_flags, g->d_red, g->d_mask, g->d_mask_c, g->d_bcount, g->d_bws,
                   g->d_members, g->d_hoff, g->d_hblob, g->d_gtab, g->d_cta_off};
  for (void* p : dptrs) {
    const unsigned char* c = static_cast<const unsigned char*>(p);
    if (p && !(g->d_arena && c >= g->d_arena && c < g->d_arena + g->arena_bytes)) cudaFree(p);
  }
  if (g->d_arena) cudaFree(g->d_arena);
  if (g->h_arena) cudaFreeHost(g->h_arena);
  if (g->ev0) cudaEventDestroy(g->ev0);
  if (g->ev1) cudaEventDestroy(g->ev1);
  delete g;
  cudaSetDevice(cur);
}

namespace gn {
gn_status configure_partition(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci);  // gn_iterate.cu
}

extern "C" gn_status gn_create(gn_graph** out, int32_t n, const int32_t* row_ptr,
                               const int32_t* col_idx, const float* w, int mem, int reorder,
                               void* stream) {
  gn_create_opts o;
  o.reorder = reorder;
  o.gather = GN_GATHER_AUTO;
  return gn_create_ex(out, n, row_ptr, col_idx, w, mem, &o, stream);
}

extern "C" int gn_gather_mode(const gn_graph* g) { return g ? g->gather : 0; }

extern "C" int gn_halo_exchange(const gn_graph* g) {
  if (!g || g->gather != GN_GATHER_HALO) return 0;
  return g->halo_push ? 2 : 1;
}

extern "C" gn_status gn_create_ex(gn_graph** out, int32_t n, const int32_t* row_ptr,
                                  const int32_t* col_idx, const float* w, int mem,
                                  const gn_create_opts* opts, void* stream) {
  using namespace gn;
  const int reorder = opts ? opts->reorder : GN_REORDER_NONE;
  const int gather = opts ? opts->gather : GN_GATHER_AUTO;
  if (!out) return fail(GN_ERR_ARG, "gn_create: out is NULL");
  *out = nullptr;
  if (gather < GN_GATHER_AUTO || gather > GN_GATHER_HALO_PUSH) return fail(GN_ERR_ARG, "gn_create: bad gather mode");
  if (n < 0 || n == INT32_MAX || !row_ptr || (!w && n > 0) || (mem != GN_HOST && mem != GN_DEVICE) ||
      reorder < GN_REORDER_NONE || reorder > GN_REORDER_DEGREE)
    return fail(GN_ERR_ARG, "gn_create: bad argument");

  gn_graph* g = new gn_graph();
  struct Guard {
    gn_graph*& g;
    ~Guard() { if (g) gn_destroy(g); }
  } guard{g};
  g->stream = (cudaStream_t)stream;
  g->io_mem = mem;
  g->n = n;
  g->reorder = reorder;
  GN_CUDA(cudaGetDevice(&g->device));
  GN_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device));

  // row_ptr on the host: structural checks and the partition need it
  std::vector<int32_t> rp(n + 1);
  if (mem == GN_HOST) {
    memcpy(rp.data(), row_ptr, sizeof(int32_t) * (n + 1));
  } else {
    GN_CUDA(cudaMemcpyAsync(rp.data(), row_ptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost,
                            g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
  }
  if (rp[0] != 0) return fail(GN_ERR_ARG, "gn_create: row_ptr[0] != 0");
  for (int i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return fail(GN_ERR_ARG, "gn_create: row_ptr decreases");
  g->nnz = rp[n];
  if (g->nnz > 0 && !col_idx) return fail(GN_ERR_ARG, "gn_create: col_idx is NULL");

  // the fixed-size buffers: one device allocation cut into 256-byte-aligned ranges, and one
  // pinned host allocation (a reordered handle also gets its permutations and the permuted
  // weights there)
  const size_t nb = sizeof(float) * std::max<int64_t>(n, 1);
  const bool reordering = reorder != GN_REORDER_NONE && n > 1;
  float* d_w_perm = nullptr;
  {
    struct Range {
      void** p;
      size_t bytes;
    };
    const Range ranges[] = {
        {(void**)&g->d_row_ptr, sizeof(int32_t) * ((size_t)n + 1)},
        {(void**)&g->d_col_idx, sizeof(int32_t) * (size_t)std::max<int64_t>(g->nnz, 1)},
        {(void**)&g->d_w, nb},
        {(void**)&g->d_v, nb},
        {(void**)&g->d_vlo, nb},
        {(void**)&g->d_ylo, nb},
        {(void**)&g->d_yexp, nb},
        {(void**)&g->d_y[0], nb},
        {(void**)&g->d_y[1], nb},
        {(void**)&g->d_x, nb},
        {(void**)&g->d_tmp, nb},
        {(void**)&g->d_bsum, sizeof(double) * 4 * 1024},
        {(void**)&g->d_io, std::max<size_t>(nb, 8 * ((size_t)n + 8))},
        {(void**)&g->d_flags, sizeof(int) * 8},
        {(void**)&g->d_info, sizeof(DevInfo)},
        {(void**)&g->d_red, sizeof(double) * 8},
        {(void**)&g->d_bar, sizeof(unsigned) * 8},
        {(void**)&g->d_mask, (size_t)std::max<int64_t>(n, 1)},
        {(void**)&g->d_mask_c, (size_t)std::max<int64_t>(n, 1)},
        {(void**)&g->d_bcount, sizeof(int) * ((size_t)n / 256 + 2)},
        {(void**)&g->d_bws, sizeof(double) * ((size_t)n / 256 + 2)},
        {(void**)&g->d_members, sizeof(int32_t) * ((size_t)std::max<int64_t>(n, 1) + 1)},
        {reordering ? (void**)&g->d_perm : nullptr, sizeof(int32_t) * (size_t)n},
        {reordering ? (void**)&g->d_iperm : nullptr, sizeof(int32_t) * (size_t)n},
        {reordering ? (void**)&d_w_perm : nullptr, nb},
    };
    auto round256 = [](size_t b) { return (b + 255) & ~(size_t)255; };
    size_t total = 0;
    for (const Range& r : ranges)
      if (r.p) total += round256(r.bytes);
    GN_CUDA(cudaMalloc(&g->d_arena, total));
    g->arena_bytes = total;
    size_t at = 0;
    for (const Range& r : ranges)
      if (r.p) {
        *r.p = g->d_arena + at;
        at += round256(r.bytes);
      }
    const size_t h_bytes = 256 + 64 + 64;  // DevInfo, 8 flags, 8 doubles
    static_assert(sizeof(DevInfo) <= 256, "DevInfo grew past its pinned slot");
    GN_CUDA(cudaMallocHost(&g->h_arena, h_bytes));
    g->h_info = reinterpret_cast<DevInfo*>(g->h_arena);
    g->h_flags = reinterpret_cast<int*>(g->h_arena + 256);
    g->h_red = reinterpret_cast<double*>(g->h_arena + 320);
  }
  GN_CUDA(cudaEventCreate(&g->ev0));
  GN_CUDA(cudaEventCreate(&g->ev1));

  cudaMemcpyKind kind = mem == GN_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  GN_CUDA(cudaMemcpyAsync(g->d_row_ptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                          g->stream));
  if (g->nnz > 0)
    GN_CUDA(cudaMemcpyAsync(g->d_col_idx, col_idx, sizeof(int32_t) * g->nnz, kind, g->stream));
  if (n > 0) GN_CUDA(cudaMemcpyAsync(g->d_w, w, sizeof(float) * n, kind, g->stream));

  // device validation: range / order / self-loops first, symmetry only on in-range data
  GN_CUDA(cudaMemsetAsync(g->d_flags, 0, sizeof(int) * 8, g->stream));
  if (n > 0) {
    k_check_rows<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, g->d_flags);
    GN_LAUNCHED();
    k_weights<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_w, g->d_v, g->d_vlo, g->d_flags);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
  }
  GN_CUDA(cudaMemcpyAsync(g->h_flags, g->d_flags, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (g->h_flags[0] & DEV_BAD_CSR) return fail(GN_ERR_ARG, "gn_create: col_idx entry out of range");
  if (g->nnz > 0) {
    k_check_symmetry<<<grid_for(g->nnz, 256), 256, 0, g->stream>>>(n, g->nnz, g->d_row_ptr,
                                                                  g->d_col_idx, g->d_flags);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
    GN_CUDA(cudaMemcpyAsync(g->h_flags, g->d_flags, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
  }
  if (g->h_flags[0] & DEV_NOT_SIMPLE)
    return fail(GN_ERR_NOT_SIMPLE, "gn_create: graph is not simple (self-loop, unsorted or duplicate "
                                   "row entries, or asymmetric adjacency)");
  if (g->h_flags[0] & DEV_BAD_WEIGHT) return fail(GN_ERR_WEIGHT, "gn_create: weight <= 0 or not finite");

  // the CSR on the host: the reordering and the per-CTA halo lists are built from it
  std::vector<int32_t> ci_host;
  const int32_t* ci_h = col_idx;
  if (mem == GN_DEVICE || g->nnz == 0) {
    ci_host.resize((size_t)std::max<int64_t>(g->nnz, 1));
    if (g->nnz > 0)
      GN_CUDA(cudaMemcpyAsync(ci_host.data(), g->d_col_idx, sizeof(int32_t) * g->nnz, cudaMemcpyDeviceToHost,
                              g->stream));
    GN_CUDA(cudaStreamSynchronize(g->stream));
    ci_h = ci_host.data();
  }

  std::unique_ptr<int32_t[]> ci_renumbered;  // the rows in the internal order, when reordered

  // optional locality reordering (internal; undone on every output)
  if (reorder != GN_REORDER_NONE && n > 1) {
    std::vector<int32_t> perm;
    bool on_device = false;  // order and renumbering done on the device (RCM in its scope)
    if (reorder == GN_REORDER_RCM) {
      gn_status st = rcm_reorder_device(g, rp, ci_renumbered, &on_device);
      if (st != GN_OK) return st;
      if (!on_device) rcm_order(n, rp, ci_h, perm);
      g->reorder_where = on_device ? GN_ORDER_FROM_DEVICE : GN_ORDER_FROM_HOST;
    } else {
      g->reorder_where = GN_ORDER_FROM_HOST;
      perm.resize(n);
      std::iota(perm.begin(), perm.end(), 0);
      std::stable_sort(perm.begin(), perm.end(),
                       [&](int a, int b) { return rp[a + 1] - rp[a] > rp[b + 1] - rp[b]; });
    }
    if (!on_device) {
      // iperm, the new row pointers and the renumbered rows, in two passes over row blocks on the
      // host threads (the blocks are the same in both passes): the first scatters iperm and sums
      // each block's degrees, the second writes each block's rows from its offset, sorted
      std::vector<int32_t> iperm(n), rp2(n + 1);
      std::unique_ptr<int32_t[]> ci2(new int32_t[(size_t)std::max<int64_t>(g->nnz, 1)]);
      std::vector<int64_t> boff(host_threads() + 1, 0);
      constexpr int kRowGrain = 4096;
      parallel_for(n, kRowGrain, [&](int lo, int hi, int t) {
        int64_t sum = 0;
        for (int r = lo; r < hi; ++r) {
          const int o = perm[r];
          iperm[o] = r;
          sum += rp[o + 1] - rp[o];
        }
        boff[t + 1] = sum;
      });
      for (size_t t = 1; t < boff.size(); ++t) boff[t] += boff[t - 1];
      parallel_for(n, kRowGrain, [&](int lo, int hi, int t) {
        int32_t at = (int32_t)boff[t];
        for (int r = lo; r < hi; ++r) {
          const int o = perm[r], d = rp[o + 1] - rp[o];
          rp2[r] = at;
          int32_t* dst = ci2.get() + at;
          for (int k = 0; k < d; ++k) dst[k] = iperm[ci_h[rp[o] + k]];
          if (d <= 32) {  // insertion sort: rows are short
            for (int k = 1; k < d; ++k) {
              const int32_t x = dst[k];
              int j = k;
              for (; j > 0 && dst[j - 1] > x; --j) dst[j] = dst[j - 1];
              dst[j] = x;
            }
          } else {
            std::sort(dst, dst + d);
          }
          at += d;
        }
      });
      rp2[n] = (int32_t)g->nnz;
      GN_CUDA(cudaMemcpyAsync(g->d_perm, perm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, g->stream));
      GN_CUDA(cudaMemcpyAsync(g->d_iperm, iperm.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, g->stream));
      GN_CUDA(cudaMemcpyAsync(g->d_row_ptr, rp2.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice,
                              g->stream));
      if (g->nnz > 0)
        GN_CUDA(cudaMemcpyAsync(g->d_col_idx, ci2.get(), sizeof(int32_t) * g->nnz, cudaMemcpyHostToDevice,
                                g->stream));
      rp.swap(rp2);
      ci_renumbered = std::move(ci2);
    }
    ci_h = ci_renumbered.get();
    float* d_w2 = d_w_perm;  // the weights in the internal order (the caller-order copy stays unused)
    k_permute_w<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_perm, g->d_w, d_w2);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
    g->d_w = d_w2;
    k_weights<<<grid_for(n, 256), 256, 0, g->stream>>>(n, g->d_w, g->d_v, g->d_vlo, g->d_flags);
    GN_LAUNCHED();
    GN_CUDA(cudaGetLastError());
  }

  g->gather = gather;
  gn_status st = configure_partition(g, rp, ci_h);
  if (st != GN_OK) return st;
  GN_CUDA(cudaStreamSynchronize(g->stream));
  *out = g;
  g = nullptr;  // disarm the guard
  return GN_OK;
}
