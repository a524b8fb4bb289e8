// gn_reorder.cu -- the reverse Cuthill-McKee vertex order on the device.
//
// The order is the host's (gn_graph.cu, rcm_order) exactly: components are started, in turn, at
// the unplaced vertex of least degree (ties by id); a breadth-first search places each vertex's
// unplaced neighbours after everything placed so far, sorted by degree (ties by adjacency order);
// the result is reversed.  Level by level that is the same as: every vertex of the next level is
// the child of its first neighbour, in queue order, in the current level, and the children of one
// parent keep the host's degree order.
//
// One thread-block cluster (kRcmC CTAs on kRcmC SMs, distributed shared memory) runs the whole
// search: a level costs three cluster barriers, and its scattered loads, claims and stores are
// shared by kRcmC SMs' memory pipelines (one SM alone is bound by the rate at which it issues
// them).  Vertex iq of a level (its index in the level's queue segment) belongs to CTA iq % kRcmC,
// slot iq / kRcmC, which holds its adjacency list in shared memory.  par[v] holds the claim on v:
// INT_MAX unreached, else the smallest queue position of a vertex that reached it (its parent);
// claims are made with atomicMin, so the first parent in queue order wins whatever the timing.
// A level takes three steps:
//   A. each CTA, a thread per own adjacency entry: is the neighbour unplaced and claimed by the
//      entry's vertex (a child), with its degree and row start; then a thread per own vertex: the
//      count and degree sum of its children, to every CTA;
//   B. every CTA scans the counts (the same scan everywhere) for the first child's queue position
//      of each vertex; a child's rank among its siblings by (degree, adjacency order) places it;
//      each child's row start and degree go to its owner CTA, and its mark to every CTA; each
//      owner lays out its next-level adjacency buffer by a scan of its vertices' degrees;
//   C. each CTA, a thread per own adjacency entry (rows read coalesced): the neighbour ids into
//      shared memory and the claims of the unplaced ones.
// Each CTA keeps a bit per vertex marking the placed ones (when it fits in shared memory), so
// that their entries need no load or claim.  A level with more vertices or entries than the
// buffers hold, a search past the level budget or a degree above the bound returns a status and
// the host computes the order itself.  Every loop is bounded by n, the capacities or the level
// budget; every exit is taken by all CTAs together, at the same point.
//
// After the search, six small kernels renumber the CSR in the new order on the device (the host
// keeps a copy for its block builder); each does nothing unless the search succeeded.
#include <cooperative_groups.h>

#include <climits>
#include <cstring>
#include <memory>

#include "gn_internal.cuh"

namespace gn {

namespace cg = cooperative_groups;

constexpr int kRcmC = 8;                // CTAs of the cluster
constexpr int kRcmThreads = 1024;
constexpr int kRcmMaxDeg = 254;         // degrees are held in bytes (0xff marks a non-child)
constexpr int kRcmMinVertices = 16384;  // below this the host search is as fast as a launch
constexpr int kRcmSlots = kRcmThreads;  // vertices of one level per CTA
constexpr int kRcmFCap = kRcmC * kRcmSlots;  // vertices of one level
constexpr int kRcmECap = 4096;          // adjacency entries of one level per CTA
constexpr int kRcmBatch = 8;            // entries per thread with loads in flight together

// dynamic shared memory of a CTA, before the placed bits
struct RcmShared {
  int adj[2][kRcmECap];        // the level's / the next level's adjacency entries of own vertices
  int seg[2][kRcmSlots];       // per own vertex: first entry in adj
  int deg[2][kRcmSlots];       // per own vertex: degree
  int row[kRcmSlots];          // per own next-level vertex: first CSR entry
  uint16_t slot[2][kRcmECap];  // per entry of adj: its own vertex
  uint8_t ek[kRcmECap];        // per entry of the level: the neighbour's degree if it is a child
                               // of the entry's vertex, else 0xff
  int erow[kRcmECap];          // per entry of the level that is a child: its first CSR entry
  int nent[2];                 // entries in adj[.]
  uint8_t cnt_c[kRcmFCap];     // per vertex of the level: children (written by its CTA into all)
  uint16_t cnt_d[kRcmFCap];    // per vertex of the level: the children's degree sum
  int offc[kRcmSlots];         // per own vertex: its first child's index in the next level
  int overflow;                // set in every CTA when a buffer would overflow
  int pad;
};
constexpr size_t kRcmSmem = (sizeof(RcmShared) + 15) & ~(size_t)15;

namespace {

// exclusive prefixes of a and b over the CTA (exactly kRcmThreads threads); s holds 64 ints
__device__ __forceinline__ int2 rcm_scan2(int a, int b, int2& total, int* s) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = a, y = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int xa = __shfl_up_sync(0xffffffffu, x, o), yb = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) {
      x += xa;
      y += yb;
    }
  }
  if (lane == 31) {
    s[wid] = x;
    s[32 + wid] = y;
  }
  __syncthreads();
  if (wid == 0) {
    int u = s[lane], v = s[32 + lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int ua = __shfl_up_sync(0xffffffffu, u, o), vb = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) {
        u += ua;
        v += vb;
      }
    }
    s[lane] = u;
    s[32 + lane] = v;
  }
  __syncthreads();
  const int2 pre = make_int2((wid ? s[wid - 1] : 0) + x - a, (wid ? s[32 + wid - 1] : 0) + y - b);
  total = make_int2(s[31], s[63]);
  __syncthreads();  // s is reused by the next call
  return pre;
}

__device__ __forceinline__ int rcm_min(int v, int* s) {
  v = __reduce_min_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  const int r = __reduce_min_sync(0xffffffffu, s[threadIdx.x & 31]);
  __syncthreads();
  return r;
}

}  // namespace

// by_deg: the vertices by (degree, id); its first n0 have degree 0.  order receives the
// Cuthill-McKee queue (not yet reversed).  bits: whether each CTA also holds the placed bits.
// Degrees are at most kRcmMaxDeg.  status (written by CTA 0): 0 done; 1 a level beyond the buffers
// or the level budget; 3 no start found although vertices remained (impossible).
__global__ void __cluster_dims__(kRcmC, 1, 1) __launch_bounds__(kRcmThreads, 1)
k_rcm(int n, const int32_t* __restrict__ rp, const int32_t* __restrict__ ci,
      const int32_t* __restrict__ by_deg, int n0, int max_levels, int bits, int32_t* par, int32_t* order,
      int* status) {
  cg::cluster_group cl = cg::this_cluster();
  extern __shared__ int4 rcm_smem[];
  RcmShared& S = *reinterpret_cast<RcmShared*>(rcm_smem);
  unsigned* placed = bits ? reinterpret_cast<unsigned*>(reinterpret_cast<char*>(rcm_smem) + kRcmSmem) : nullptr;
  __shared__ int s[64];
  const int tid = threadIdx.x, rank = (int)cl.block_rank();
  auto is_placed = [placed](int v) { return placed && (placed[v >> 5] >> (v & 31) & 1u); };
  auto mark_here = [placed](int v) {
    if (placed) atomicOr(placed + (v >> 5), 1u << (v & 31));
  };
  auto mark_all = [&](int v) {
    if (placed)
      for (int r = 0; r < kRcmC; ++r) atomicOr(cl.map_shared_rank(placed, r) + (v >> 5), 1u << (v & 31));
  };

  if (tid == 0) {
    S.nent[0] = S.nent[1] = 0;
    S.overflow = 0;
  }
  for (int i = rank * kRcmThreads + tid; i < n; i += kRcmC * kRcmThreads) par[i] = INT_MAX;
  if (placed)
    for (int i = tid; i < (n + 31) / 32; i += kRcmThreads) placed[i] = 0u;
  cl.sync();
  // isolated vertices are components of their own, started in by_deg order before any other
  for (int i = tid; i < n0; i += kRcmThreads) {
    const int v = by_deg[i];
    mark_here(v);
    if (i % kRcmC == rank) {
      order[i] = v;
      par[v] = -1;
    }
  }
  cl.sync();

  int filled = n0, cursor = n0, levels = 0, cur = 0;
  while (filled < n) {
    // the next start, found alike by every CTA: the first vertex of by_deg past the cursor that is
    // still unreached (a vertex is placed exactly when its claim is not INT_MAX: no claim is
    // pending between components)
    int first = INT_MAX;
    while (cursor < n) {
      const int i = cursor + tid;
      bool open = false;
      if (i < n) {
        const int v = by_deg[i];
        open = placed ? !is_placed(v) : __ldcg(par + v) == INT_MAX;
      }
      first = rcm_min(open ? i : INT_MAX, s);
      if (first != INT_MAX) break;
      cursor += kRcmThreads;
    }
    if (first == INT_MAX) {
      if (rank == 0 && tid == 0) *status = 3;
      return;
    }
    if (++levels > max_levels) {
      if (rank == 0 && tid == 0) *status = 1;
      return;
    }
    cursor = first + 1;
    const int s0 = by_deg[first];
    if (tid == 0) {
      mark_here(s0);
      S.nent[cur] = 0;
    }
    if (rank == 0) {  // the start is vertex 0 of its level: CTA 0, slot 0
      const int k0 = rp[s0], d0 = rp[s0 + 1] - k0;  // 1 <= d0 <= kRcmMaxDeg
      __syncthreads();  // the start's mark before its neighbours are tested
      if (tid == 0) {
        order[filled] = s0;
        atomicMin(par + s0, -1);
        S.seg[cur][0] = 0;
        S.deg[cur][0] = d0;
        S.nent[cur] = d0;
      }
      for (int k = tid; k < d0; k += kRcmThreads) {
        const int x = ci[k0 + k];
        S.adj[cur][k] = x;
        S.slot[cur][k] = 0;
        if (!is_placed(x)) atomicMin(par + x, filled);
      }
    }
    cl.sync();

    int fs = filled, F = 1;  // this level: queue positions [fs, fs + F)
    while (F > 0) {
      if (++levels > max_levels) {
        if (rank == 0 && tid == 0) *status = 1;
        return;
      }
      const int fe = fs + F, nxt = cur ^ 1;
      // A1. own entries of the level, consecutive entries on consecutive threads: is the neighbour
      // unplaced and claimed by the entry's vertex (a child), and its degree and first entry (loaded
      // with the claim, not after it)
      const int ownA = S.nent[cur];
      for (int b0 = 0; b0 < ownA; b0 += kRcmThreads * kRcmBatch) {
        int w[kRcmBatch], p[kRcmBatch], pv[kRcmBatch], r0[kRcmBatch], r1[kRcmBatch];
#pragma unroll
        for (int u = 0; u < kRcmBatch; ++u) {
          const int e = b0 + u * kRcmThreads + tid;
          w[u] = -1;
          if (e < ownA) {
            const int x = S.adj[cur][e];
            if (is_placed(x)) {
              S.ek[e] = 0xff;
            } else {
              w[u] = x;
              p[u] = fs + S.slot[cur][e] * kRcmC + rank;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kRcmBatch; ++u)
          if (w[u] >= 0) {
            pv[u] = __ldcg(par + w[u]);
            r0[u] = rp[w[u]];
            r1[u] = rp[w[u] + 1];
          }
#pragma unroll
        for (int u = 0; u < kRcmBatch; ++u) {
          const int e = b0 + u * kRcmThreads + tid;
          if (w[u] < 0) continue;
          if (pv[u] == p[u]) {
            S.ek[e] = (uint8_t)(r1[u] - r0[u]);
            S.erow[e] = r0[u];
          } else {
            S.ek[e] = 0xff;
          }
        }
      }
      __syncthreads();
      // A2. per own vertex of the level, its children's count and degree sum, into every CTA
      const int i = tid * kRcmC + rank;  // this thread's vertex of the level
      if (i < F) {
        int c = 0, dsum = 0;
        const int e0 = S.seg[cur][tid], e1 = e0 + S.deg[cur][tid];
        for (int e = e0; e < e1; ++e) {
          const int d = S.ek[e];
          if (d == 0xff) continue;
          ++c;
          dsum += d;
        }
        for (int r = 0; r < kRcmC; ++r) {
          RcmShared* P = cl.map_shared_rank(&S, r);
          P->cnt_c[i] = (uint8_t)c;
          P->cnt_d[i] = (uint16_t)dsum;
        }
      }
      cl.sync();
      // B. every CTA scans the counts alike: the children's indices in the next level, and the
      // next level's size
      int Fn;
      {
        constexpr int E = kRcmFCap / kRcmThreads;  // counts per thread
        const int i0 = tid * E;
        int sc = 0, sd = 0;
#pragma unroll
        for (int t = 0; t < E; ++t)
          if (i0 + t < F) {
            sc += S.cnt_c[i0 + t];
            sd += S.cnt_d[i0 + t];
          }
        int2 tot;
        const int2 off = rcm_scan2(sc, sd, tot, s);
        int oc = off.x;
#pragma unroll
        for (int t = 0; t < E; ++t)
          if (i0 + t < F) {
            if ((i0 + t) % kRcmC == rank) S.offc[(i0 + t) / kRcmC] = oc;
            oc += S.cnt_c[i0 + t];
          }
        Fn = tot.x;
      }
      __syncthreads();
      if (Fn > kRcmFCap) {  // the same decision in every CTA
        if (rank == 0 && tid == 0) *status = 1;
        return;
      }
      // the children into their owners (row start and degree), a thread per own entry that is a
      // child: its index among its parent's children by (degree, adjacency order)
      for (int e = tid; e < ownA; e += kRcmThreads) {
        const int d = S.ek[e];
        if (d == 0xff) continue;
        const int t = S.slot[cur][e], e0 = S.seg[cur][t], e1 = e0 + S.deg[cur][t];
        int rank_in = 0;
        for (int f = e0; f < e1; ++f) {
          const int df = S.ek[f];
          rank_in += df != 0xff && (df < d || (df == d && f < e));
        }
        // a placed vertex keeps its claim: no later level's position can equal it
        const int iq = S.offc[t] + rank_in, w = S.adj[cur][e];
        order[fe + iq] = w;
        mark_all(w);
        RcmShared* P = cl.map_shared_rank(&S, iq % kRcmC);
        P->deg[nxt][iq / kRcmC] = d;
        P->row[iq / kRcmC] = S.erow[e];
      }
      cl.sync();
      // each CTA lays out its own next-level vertices' entries (a scan of their degrees); a CTA
      // whose entries would overflow its buffer skips step C and sets the flag in every CTA
      const int Fo = (Fn - rank + kRcmC - 1) / kRcmC;  // own next-level vertices
      int own;
      {
        const int d = tid < Fo ? S.deg[nxt][tid] : 0;
        int2 tot;
        const int e = rcm_scan2(d, 0, tot, s).x;
        own = tot.x;
        if (own <= kRcmECap && tid < Fo) {
          S.seg[nxt][tid] = e;
          for (int k = 0; k < d; ++k) S.slot[nxt][e + k] = (uint16_t)tid;
        }
        if (own > kRcmECap) {
          if (tid == 0)
            for (int r = 0; r < kRcmC; ++r) cl.map_shared_rank(&S, r)->overflow = 1;
          own = 0;
        }
        if (tid == 0) S.nent[nxt] = own;
        __syncthreads();
      }
      // C. own next-level entries, consecutive entries on consecutive threads: the neighbour ids
      // into shared memory and the claims of the unplaced ones
      for (int b0 = 0; b0 < own; b0 += kRcmThreads * kRcmBatch) {
        int x[kRcmBatch], q[kRcmBatch];
#pragma unroll
        for (int u = 0; u < kRcmBatch; ++u) {
          const int e = b0 + u * kRcmThreads + tid;
          q[u] = -1;
          if (e < own) {
            const int t = S.slot[nxt][e];
            q[u] = fe + t * kRcmC + rank;
            x[u] = ci[S.row[t] + (e - S.seg[nxt][t])];
          }
        }
#pragma unroll
        for (int u = 0; u < kRcmBatch; ++u)
          if (q[u] >= 0) {
            S.adj[nxt][b0 + u * kRcmThreads + tid] = x[u];
            if (!is_placed(x[u])) atomicMin(par + x[u], q[u]);
          }
      }
      cl.sync();
      if (S.overflow) {  // set in every CTA before the barrier
        if (rank == 0 && tid == 0) *status = 1;
        return;
      }
      cur = nxt;
      fs = fe;
      F = Fn;
    }
    filled = fs;
  }
  if (rank == 0 && tid == 0) *status = 0;
}

// ------------------------------------------------------------------------------------------
// renumbering in the new order, on the device, right after the search: every kernel first reads
// the search's status and does nothing unless it succeeded (no host round trip in between)

constexpr int kRnTile = 4096;  // row degrees per block of the scan (1024 threads x 4)

// perm[r] = order[n - 1 - r] (the reversal), iperm, and the degrees in the new order
__global__ void k_rn_perm(int n, const int* __restrict__ status, const int32_t* __restrict__ order,
                          const int32_t* __restrict__ rp, int32_t* __restrict__ perm, int32_t* __restrict__ iperm,
                          int32_t* __restrict__ deg) {
  if (*status != 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int o = order[n - 1 - r];
  perm[r] = o;
  iperm[o] = r;
  deg[r] = rp[o + 1] - rp[o];
}

// sum of each tile of kRnTile degrees
__global__ void __launch_bounds__(1024) k_rn_tile_sums(int n, const int* __restrict__ status,
                                                       const int32_t* __restrict__ deg, int32_t* __restrict__ tsum) {
  if (*status != 0) return;
  __shared__ int s[32];
  int v = 0;
  for (int i = blockIdx.x * kRnTile + threadIdx.x; i < min(n, (blockIdx.x + 1) * kRnTile); i += blockDim.x)
    v += deg[i];
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    const int t = __reduce_add_sync(0xffffffffu, s[threadIdx.x]);
    if (threadIdx.x == 0) tsum[blockIdx.x] = t;
  }
}

// exclusive prefix of the tile sums, in place (one CTA, any number of tiles)
__global__ void __launch_bounds__(1024) k_rn_tile_scan(int ntiles, const int* __restrict__ status,
                                                       int32_t* __restrict__ tsum) {
  if (*status != 0) return;
  __shared__ int s[64];
  int carry = 0;
  for (int base = 0; base < ntiles; base += kRcmThreads) {
    const int i = base + threadIdx.x;
    const int v = i < ntiles ? tsum[i] : 0;
    int2 tot;
    const int pre = rcm_scan2(v, 0, tot, s).x;
    if (i < ntiles) tsum[i] = carry + pre;
    carry += tot.x;
  }
}

// the new row pointers: each tile's exclusive prefix from its offset; rp2[n] = nnz
__global__ void __launch_bounds__(1024) k_rn_rowptr(int n, int32_t nnz, const int* __restrict__ status,
                                                    const int32_t* __restrict__ deg, const int32_t* __restrict__ toff,
                                                    int32_t* __restrict__ rp2) {
  if (*status != 0) return;
  __shared__ int s[64];
  constexpr int E = kRnTile / 1024;
  const int i0 = blockIdx.x * kRnTile + threadIdx.x * E;
  int d[E], sum = 0;
#pragma unroll
  for (int t = 0; t < E; ++t) {
    d[t] = i0 + t < n ? deg[i0 + t] : 0;
    sum += d[t];
  }
  int2 tot;
  int at = toff[blockIdx.x] + rcm_scan2(sum, 0, tot, s).x;
#pragma unroll
  for (int t = 0; t < E; ++t)
    if (i0 + t < n) {
      rp2[i0 + t] = at;
      at += d[t];
    }
  if (blockIdx.x == 0 && threadIdx.x == 0) rp2[n] = nnz;
}

// the rows in the new order, their entries renumbered and sorted (rows are short: the search
// runs only for degrees up to kRcmMaxDeg)
__global__ void k_rn_rows(int n, const int* __restrict__ status, const int32_t* __restrict__ rp,
                          const int32_t* __restrict__ ci, const int32_t* __restrict__ perm,
                          const int32_t* __restrict__ iperm, const int32_t* __restrict__ rp2, int32_t* __restrict__ ci2) {
  if (*status != 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int o = perm[r], a = rp[o], d = rp[o + 1] - a;
  int32_t* dst = ci2 + rp2[r];
  for (int k = 0; k < d; ++k) {
    const int32_t x = iperm[ci[a + k]];
    int j = k;
    for (; j > 0 && dst[j - 1] > x; --j) dst[j] = dst[j - 1];
    dst[j] = x;
  }
}

// the renumbered CSR over the handle's (caller-order) one
__global__ void k_rn_copy(int n, int64_t nnz, const int* __restrict__ status, const int32_t* __restrict__ rp2,
                          const int32_t* __restrict__ ci2, int32_t* __restrict__ rp, int32_t* __restrict__ ci) {
  if (*status != 0) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) rp[i] = rp2[i];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nnz; i += stride) ci[i] = ci2[i];
}

// Reverse Cuthill-McKee order of the caller-order CSR already on the device (g->d_row_ptr,
// g->d_col_idx, validated), and the renumbering in it, all on the device.  On success (*done):
// g->d_perm and g->d_iperm hold the order (perm[r] = the caller's vertex placed r-th after the
// reversal), g->d_row_ptr and g->d_col_idx the renumbered CSR (rows sorted), and rp and *ci_new
// the same CSR on the host.  *done is false (nothing changed) when the graph is outside the
// search's scope (few vertices, a degree above kRcmMaxDeg), the cluster cannot be launched, or
// the search stopped (a level past the buffers or the level budget); the host then computes the
// same order and renumbers.
gn_status rcm_reorder_device(gn_graph* g, std::vector<int32_t>& rp, std::unique_ptr<int32_t[]>& ci_new,
                             bool* done) {
  *done = false;
  const int n = g->n;
  const int64_t nnz = g->nnz;
  if (n < kRcmMinVertices) return GN_OK;
  // degrees and a stable counting sort by degree, split over the host threads
  const int nt = std::max(1, std::min(host_threads(), n / 4096));
  std::vector<int> tmax(nt, 0);
  parallel_for(n, (n + nt - 1) / nt, [&](int lo, int hi, int t) {
    int m = 0;
    for (int i = lo; i < hi; ++i) m = std::max(m, rp[i + 1] - rp[i]);
    tmax[t] = m;
  });
  const int dmax = *std::max_element(tmax.begin(), tmax.end());
  if (dmax > kRcmMaxDeg) return GN_OK;
  std::vector<int32_t> cnt((size_t)nt * (dmax + 1), 0), by_deg(n);
  parallel_for(n, (n + nt - 1) / nt, [&](int lo, int hi, int t) {
    int32_t* c = cnt.data() + (size_t)t * (dmax + 1);
    for (int i = lo; i < hi; ++i) ++c[rp[i + 1] - rp[i]];
  });
  int32_t run = 0;
  for (int d = 0; d <= dmax; ++d)
    for (int t = 0; t < nt; ++t) {
      const int32_t c = cnt[(size_t)t * (dmax + 1) + d];
      cnt[(size_t)t * (dmax + 1) + d] = run;
      run += c;
    }
  parallel_for(n, (n + nt - 1) / nt, [&](int lo, int hi, int t) {
    int32_t* c = cnt.data() + (size_t)t * (dmax + 1);
    for (int i = lo; i < hi; ++i) by_deg[c[rp[i + 1] - rp[i]]++] = i;
  });
  int n0 = 0;
  while (n0 < n && rp[by_deg[n0] + 1] == rp[by_deg[n0]]) ++n0;

  // the placed-vertex bits when they fit beside the level buffers (1 KB for the static arrays)
  const size_t bit_bytes = sizeof(unsigned) * (((size_t)n + 31) / 32);
  int optin = 0;
  GN_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device));
  const int bits = kRcmSmem + bit_bytes + 1024 <= (size_t)optin;
  const size_t smem = kRcmSmem + (bits ? bit_bytes : 0);
  GN_CUDA(cudaFuncSetAttribute(k_rcm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int clusters = 0;
  {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kRcmC);
    cfg.blockDim = dim3(kRcmThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = g->stream;
    if (cudaOccupancyMaxActiveClusters(&clusters, k_rcm, &cfg) != cudaSuccess) {
      (void)cudaGetLastError();
      clusters = 0;
    }
  }
  if (clusters < 1) return GN_OK;

  // scratch: by_deg, par, order, degrees, new row pointers, tile sums, new rows, status
  const int ntiles = (n + kRnTile - 1) / kRnTile;
  const size_t words = 4 * (size_t)n + ((size_t)n + 1) + (size_t)ntiles + (size_t)std::max<int64_t>(nnz, 1) + 1;
  int32_t* scratch = nullptr;
  GN_CUDA(cudaMalloc(&scratch, sizeof(int32_t) * words));
  struct Free {
    int32_t* p;
    ~Free() { cudaFree(p); }
  } free_scratch{scratch};
  int32_t* d_by_deg = scratch;
  int32_t* d_par = d_by_deg + n;
  int32_t* d_order = d_par + n;
  int32_t* d_deg = d_order + n;
  int32_t* d_rp2 = d_deg + n;
  int32_t* d_tsum = d_rp2 + ((size_t)n + 1);
  int32_t* d_ci2 = d_tsum + ntiles;
  int* d_status = d_ci2 + std::max<int64_t>(nnz, 1);
  GN_CUDA(cudaMemcpyAsync(d_by_deg, by_deg.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaMemsetAsync(d_status, 0xff, sizeof(int), g->stream));
  // the search stops paying once its levels cost more than the host's per-vertex work
  const int max_levels = std::max(2048, n / 32);
  k_rcm<<<kRcmC, kRcmThreads, smem, g->stream>>>(n, g->d_row_ptr, g->d_col_idx, d_by_deg, n0, max_levels, bits,
                                                 d_par, d_order, d_status);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  const unsigned gn_ = (unsigned)((n + 255) / 256);
  k_rn_perm<<<gn_, 256, 0, g->stream>>>(n, d_status, d_order, g->d_row_ptr, g->d_perm, g->d_iperm, d_deg);
  GN_LAUNCHED();
  k_rn_tile_sums<<<ntiles, 1024, 0, g->stream>>>(n, d_status, d_deg, d_tsum);
  GN_LAUNCHED();
  k_rn_tile_scan<<<1, kRcmThreads, 0, g->stream>>>(ntiles, d_status, d_tsum);
  GN_LAUNCHED();
  k_rn_rowptr<<<ntiles, 1024, 0, g->stream>>>(n, (int32_t)nnz, d_status, d_deg, d_tsum, d_rp2);
  GN_LAUNCHED();
  k_rn_rows<<<gn_, 256, 0, g->stream>>>(n, d_status, g->d_row_ptr, g->d_col_idx, g->d_perm, g->d_iperm, d_rp2,
                                        d_ci2);
  GN_LAUNCHED();
  k_rn_copy<<<std::min<unsigned>(gn_, 1024u), 256, 0, g->stream>>>(n, nnz, d_status, d_rp2, d_ci2, g->d_row_ptr,
                                                                  g->d_col_idx);
  GN_LAUNCHED();
  GN_CUDA(cudaGetLastError());
  int status = -1;
  GN_CUDA(cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  if (status != 0) return GN_OK;
  // the renumbered CSR on the host too (the halo blocks are built from it)
  std::vector<int32_t> rp2(n + 1);
  std::unique_ptr<int32_t[]> ci2(new int32_t[(size_t)std::max<int64_t>(nnz, 1)]);
  GN_CUDA(cudaMemcpyAsync(rp2.data(), d_rp2, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToHost, g->stream));
  if (nnz > 0)
    GN_CUDA(cudaMemcpyAsync(ci2.get(), d_ci2, sizeof(int32_t) * (size_t)nnz, cudaMemcpyDeviceToHost, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  rp.swap(rp2);
  ci_new = std::move(ci2);
  *done = true;
  return GN_OK;
}

}  // namespace gn
