// gn_halo.cu -- the halo gather mode of the persistent WRGN kernel.
//
// Each CTA owns a contiguous range of rows for the whole run and keeps everything it needs
// in shared memory:
//   s_all  = [ own weighted states y_i (hi parts) | external halo values | 32 zeros ]
//   a packed per-CTA block (built once on the host): the light rows in SELL-32 slices
//   (32 rows per slice, a lane per row, 16-bit local ids into s_all packed four per lane in
//   8-byte words, rows sorted interior-first then by degree; each column is one gather
//   instruction and touches 32 distinct banks, see color_slice), the heavy rows cut into
//   chunks of at most 256 entries
//   (a warp per chunk; a row's chunk sums are added in chunk order, so the result does not
//   depend on which warp took which chunk) and the CTA's send list.
//
// Two ways to exchange the halo, chosen per graph when the blocks are built:
//  * pull: each CTA writes its new states to the global state vector and, the next
//    iteration, gathers its halo from there with one 4-byte cp.async per value (the block
//    holds the list of external ids).  Cheap when a CTA's halo is dense in memory (a
//    bandwidth-reducing order puts a CTA's external neighbours in a few long runs).
//  * push, by inboxes: every CTA c has a contiguous inbox in global memory holding the
//    states of its external neighbours in the order of its halo (sorted by vertex id, so the
//    vertices of one owner CTA form one run).  After its update, each CTA writes its new
//    states into the runs it owns in the other CTAs' inboxes: the send list, pieces of at
//    most 128 consecutive inbox slots, a warp per piece, so the stores are coalesced.  The
//    next iteration fetches the whole inbox with one bulk copy (cp.async.bulk, completion
//    counted on an mbarrier).  Two inbox buffers alternate.  Pays off when halos are
//    scattered (a few values per 32-byte sector), where per-value gathers are bound by the
//    number of sectors each SM has in flight.
//
// One iteration (r = k - k_start):
//   1. the halo, asynchronously: pull cp.asyncs, or the bulk copy of inbox[r % 2]
//   2. row sums of the interior slices (only own rows: no wait) while the halo flies
//   3. wait for the halo; row sums of the boundary slices and of the heavy-row chunks (one
//      work list over the warps), then the heavy rows' chunk sums
//   4. the update (gn_iter_common.cuh) and the stop-test partials
//   5. push: the send list into inbox[(r + 1) % 2]
//   6. the synchronisation: a bounded grid barrier, or (neighbour synchronisation) a release
//      store of the CTA's completed-iteration count, with a grid-wide wait only at the stop
//      test
// A prologue writes the starting states into inbox[0] (push).
//
// Neighbour synchronisation.  A CTA's halo for iteration r is written by the CTAs owning it
// (its dependency list) in iteration r - 1, so before step 1 warp 0 waits for those CTAs'
// flags only.  The relation is symmetric (the graph is undirected), which also makes the
// double buffers safe: a CTA overwrites a buffer its dependents read in iteration r - 1 only
// after it has seen that they completed it.
#include <algorithm>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "gn_iter_common.cuh"

namespace gn {

// header of a CTA block (int32 words), followed by 16-byte aligned sections
struct HaloHeader {
  int ns_int;      // interior slices (every row's neighbours are own rows)
  int ns;          // all slices
  int nheavy;      // heavy rows
  int lx;          // external halo length
  int sell_len;    // SELL entries (with padding)
  int heavy_len;   // local ids of the heavy rows
  int zero_id;     // local id of the first of 32 zero slots, one per bank (padding)
  int inbox_off;   // float offset of this CTA's inbox in one inbox buffer (multiple of 4)
  int off_meta;    // byte offsets of the sections from the block start
  int off_srow;
  int off_sell;
  int off_hmeta;
  int off_hl;
  int bytes;       // block size (multiple of 16)
  int ndep;        // CTAs owning external neighbours (the dependency list)
  int off_dep;
  int nchunk;      // heavy-row chunks
  int off_hchunk;  // (entry offset into hl, count) per chunk
  int off_hpart;   // float per chunk: its sum of this iteration
  int npiece;      // send-list pieces
  int off_piece;   // int4 per piece: (first inbox slot, length, first source, 0)
  int off_src;     // uint16 per sent value: the own row it comes from
  int off_x;       // pull: int32 per halo value, its vertex id
  int pad0;
};

static constexpr int kHeavyHalo = 64;    // rows with more entries are cut into chunks
static constexpr int kHeavyChunk = 256;  // entries per chunk (8 per lane)
static constexpr int kSendPiece = 128;   // inbox slots per send piece

// SELL-32 slice s: warp per slice, lane per row.  A slice's width is a multiple of 4 and each
// lane's local ids come four at a time in one 8-byte word (layout [k/4][lane]).
__device__ __forceinline__ void sum_slice(int s, const int2* __restrict__ meta, const short* __restrict__ srow,
                                          const uint16_t* __restrict__ sell, const float* __restrict__ s_all,
                                          float* __restrict__ s_sum) {
  const int lane = threadIdx.x & 31;
  const int2 m = meta[s];  // (entry offset, width): width % 4 == 0, offset % 128 == 0
  const uint2* col = reinterpret_cast<const uint2*>(sell + m.x) + lane;
  float a0 = 0.0f, a1 = 0.0f;
  for (int q = 0; q < (m.y >> 2); ++q) {
    const uint2 ids = col[q * 32];
    a0 += s_all[ids.x & 0xffffu];
    a1 += s_all[ids.x >> 16];
    a0 += s_all[ids.y & 0xffffu];
    a1 += s_all[ids.y >> 16];
  }
  const int r = srow[s * 32 + lane];
  if (r >= 0) s_sum[r] = a0 + a1;
}

// heavy-row chunk: entries [a, a + cnt) of hl, lane-strided with four independent sums, then
// a butterfly over the warp (fixed order); lane 0 stores the chunk's sum
__device__ __forceinline__ void sum_chunk(int2 ch, const uint16_t* __restrict__ hl,
                                          const float* __restrict__ s_all, float* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
  int e = ch.x + lane;
  const int end = ch.x + ch.y;
  for (; e + 96 < end; e += 128) {
    a0 += s_all[hl[e]];
    a1 += s_all[hl[e + 32]];
    a2 += s_all[hl[e + 64]];
    a3 += s_all[hl[e + 96]];
  }
  for (; e < end; e += 32) a0 += s_all[hl[e]];
  float acc = (a0 + a1) + (a2 + a3);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) *out = acc;
}

// pull: one halo value, global -> shared, asynchronously
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}

// push: the send list, own states (s_all) into the other CTAs' inboxes, a warp per piece of
// at most 128 slots; each lane's (up to four) source reads are issued together
__device__ __forceinline__ void push_states(const int4* __restrict__ piece, int npiece,
                                            const uint16_t* __restrict__ src, const float* __restrict__ s_all,
                                            float* __restrict__ inbox) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int q = warp; q < npiece; q += nwarps) {
    const int4 pc = piece[q];
    int id[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) id[u] = lane + 32 * u < pc.y ? src[pc.z + lane + 32 * u] : -1;
    float val[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) val[u] = id[u] >= 0 ? s_all[id[u]] : 0.0f;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (id[u] >= 0) inbox[pc.x + lane + 32 * u] = val[u];
  }
}

// ---- bulk copy with mbarrier completion (TMA, non-tensor form)
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// thread 0: order the other CTAs' inbox writes (generic proxy, acquired at the last
// synchronisation) before the async-proxy read of the copy, announce the bytes, start the
// copy.  This CTA's own reads of the halo slots precede the copy through the bar.syncs since.
__device__ __forceinline__ void bulk_fetch(float* s_dst, const float* g_src, unsigned bytes, uint64_t* bar) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  const unsigned d = (unsigned)__cvta_generic_to_shared(s_dst);
  asm volatile("fence.proxy.async.global;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(d),
               "l"(g_src), "r"(bytes), "r"(b)
               : "memory");
}
// bounded wait for phase `parity` of the mbarrier; false if the limit was hit
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, long long limit) {
  const unsigned b = (unsigned)__cvta_generic_to_shared(bar);
  for (long long i = 0; i <= limit; ++i) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// REG: a CTA owns at most 2 * kThreads rows and each thread keeps its (at most two) rows'
// state in registers across iterations; only y (for the neighbour sums) goes to shared memory.
// PUSH: the halo exchange by inboxes, else pull.
template <bool REG, bool PUSH>
__global__ void __launch_bounds__(kThreads, 1) k_gn_halo(const IterParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TailShared T;
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ int s_dep_ok;
  const int R = P.rows_pad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int b = blockIdx.x;
  const int rb = P.part[b], nr = P.part[b + 1] - rb;

  // a failed start-state validation (written before the launch) ends the run at once
  if (dev::ld_relaxed_int(P.status) != 0) return;

  float* s_all = reinterpret_cast<float*>(smem);
  const int nall = R + P.halo_pad + 32;
  RowArrays S;
  S.yh = s_all;
  S.sum = s_all + nall;
  S.yl = S.sum + R;
  S.x = S.yl + R;
  S.vh = S.x + R;
  S.vl = S.vh + R;
  unsigned char* blk = reinterpret_cast<unsigned char*>(S.vl + R);
  // copy this CTA's packed block (16-byte words)
  {
    const int64_t o0 = P.hoff[b];
    const int nbytes = (int)(P.hoff[b + 1] - o0);
    const int4* src = reinterpret_cast<const int4*>(P.hblob + o0);
    int4* dst = reinterpret_cast<int4*>(blk);
    for (int t = tid; t < nbytes / 16; t += blockDim.x) dst[t] = src[t];
  }
  // own rows: registers (REG) or shared memory
  dev::f2 ry[2], rv[2];
  float rx[2], rw[2];
  if (REG) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * kThreads;
      const bool in = i < nr;
      // a row past the CTA's end is a fixed point y = x = 1 (never a safe division)
      ry[j] = in ? dev::f2{P.y0[rb + i], P.ylo[rb + i]} : dev::f2{1.0f, 0.0f};
      rv[j] = in ? dev::f2{P.v[rb + i], P.vlo[rb + i]} : dev::f2{1.0f, 0.0f};
      rx[j] = in ? P.x[rb + i] : 0.0f;
      rw[j] = in ? P.w[rb + i] : 0.0f;
      if (in) S.yh[i] = ry[j].hi;
    }
  } else {
    for (int i = tid; i < nr; i += blockDim.x) {
      S.vh[i] = P.v[rb + i];
      S.vl[i] = P.vlo[rb + i];
      S.yh[i] = P.y0[rb + i];
      S.yl[i] = P.ylo[rb + i];
      S.x[i] = P.x[rb + i];
    }
  }
  if (tid == 0) mbar_init(&s_bar, 1);
  __syncthreads();
  const HaloHeader H = *reinterpret_cast<const HaloHeader*>(blk);
  const int2* __restrict__ meta = reinterpret_cast<const int2*>(blk + H.off_meta);
  const short* __restrict__ srow = reinterpret_cast<const short*>(blk + H.off_srow);
  const uint16_t* __restrict__ sell = reinterpret_cast<const uint16_t*>(blk + H.off_sell);
  const int* __restrict__ hmeta = reinterpret_cast<const int*>(blk + H.off_hmeta);
  const uint16_t* __restrict__ hl = reinterpret_cast<const uint16_t*>(blk + H.off_hl);
  const int* __restrict__ deps = reinterpret_cast<const int*>(blk + H.off_dep);
  const int2* __restrict__ hchunk = reinterpret_cast<const int2*>(blk + H.off_hchunk);
  float* __restrict__ hpart = reinterpret_cast<float*>(blk + H.off_hpart);
  const int4* __restrict__ piece = reinterpret_cast<const int4*>(blk + H.off_piece);
  const uint16_t* __restrict__ ssrc = reinterpret_cast<const uint16_t*>(blk + H.off_src);
  const int* __restrict__ xlist = reinterpret_cast<const int*>(blk + H.off_x);
  if (tid < 32) s_all[H.zero_id + tid] = 0.0f;  // one zero slot per bank (padding)
  set_gamma(P, P.k_start, T);
  float* s_halo = s_all + R;
  const float th_lo = (float)P.theta, th_hi = (float)(1.0 - P.theta);
  const unsigned halo_bytes = (unsigned)((H.lx + 3) & ~3) * 4u;

  unsigned long long hits = 0;
  int parity = 0, slot = 0, stop = 0;
  unsigned nbar = 0;
  int nchk = 0;  // checks so far (grid mode: selects the check word)
  unsigned mphase = 0;  // parity of the mbarrier phase the next copy completes
  int k = P.k_start;

  // prologue: the starting states into inbox[0] (push), then every CTA's halo is complete
  if (PUSH) push_states(piece, H.npiece, ssrc, s_all, P.inbox);
  if (P.iterflag) {
    if (publish_and_stop(P, false, slot, false, dev::f2{0.0f, 0.0f}, k - 1, T) == 2) stop = 2;
  } else {
    ++nbar;
    if (!dev::grid_barrier(P.bar, nbar * (unsigned)P.nblocks + (P.unreachable ? 1u : 0u), P.status,
                           P.spin_limit))
      stop = 2;
  }
  // neighbour synchronisation: whether every CTA is known to have completed the pushes of
  // iteration k - 1 (after a check); the first iteration waits for the prologue's pushes
  bool synced = false;
  bool fail = false;

  for (; stop != 2 && k < P.k_end; ++k) {
    const int r = k - P.k_start;
    const dev::f2 gam = {T.gh, T.gl};
    const float2 gnext = gamma_fetch(P, k + 1);
    const float* inbox_in = PUSH ? P.inbox + (size_t)(r & 1) * (size_t)P.inbox_len : nullptr;
    float* inbox_out = PUSH ? P.inbox + (size_t)((r + 1) & 1) * (size_t)P.inbox_len : nullptr;
    const float* __restrict__ yin = parity ? P.y1 : P.y0;  // pull
    float* __restrict__ yout = parity ? P.y0 : P.y1;

    // 0. neighbour synchronisation: the dependencies' iteration r - 1 (their pushes)
    if (P.iterflag && !synced) {
      if (warp == 0) {
        const bool ok = dev::wait_flags_warp(P.iterflag, deps, H.ndep, (unsigned)r + 1u + (P.unreachable ? 1u : 0u),
                                             P.status, P.spin_limit);
        if (lane == 0) s_dep_ok = ok;
      }
      __syncthreads();
      fail = !s_dep_ok;
    }
    // 1. the halo, asynchronously
    if (PUSH) {
      if (tid == 0 && H.lx > 0 && !fail) bulk_fetch(s_halo, inbox_in + H.inbox_off, halo_bytes, &s_bar);
    } else {
      for (int t = tid; t < H.lx; t += blockDim.x) cp_async4(&s_halo[t], yin + xlist[t]);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // 2. interior rows need only own values
    for (int s = warp; s < H.ns_int; s += nwarps) sum_slice(s, meta, srow, sell, s_all, S.sum);
    // 3. boundary rows and heavy chunks after the halo has landed
    if (PUSH) {
      if (H.lx > 0 && !fail) {
        if (!mbar_wait(&s_bar, mphase, P.spin_limit)) {
          fail = true;
          if (lane == 0) atomicOr(P.status, DEV_TIMEOUT);
        }
        mphase ^= 1u;
      }
    } else {
      asm volatile("cp.async.wait_all;" ::: "memory");
    }
    __syncthreads();
    {
      // one round-robin over the warps of [boundary slices | heavy chunks], as two loops (a
      // branch inside the slice loop costs the slices more than the split does)
      const int nsb = H.ns - H.ns_int;
      for (int it = warp; it < nsb; it += nwarps) sum_slice(H.ns_int + it, meta, srow, sell, s_all, S.sum);
      if (H.nchunk)  // CTA-uniform
        for (int c = (warp - nsb % nwarps + nwarps) % nwarps; c < H.nchunk; c += nwarps)
          sum_chunk(hchunk[c], hl, s_all, hpart + c);
    }
    __syncthreads();
    if (H.nheavy) {  // CTA-uniform
      for (int h = tid; h < H.nheavy; h += blockDim.x) {
        const int rr = hmeta[3 * h], c0 = hmeta[3 * h + 1], nc = hmeta[3 * h + 2];
        float acc = 0.0f;
        for (int q = 0; q < nc; ++q) acc += hpart[c0 + q];
        S.sum[rr] = acc;
      }
      __syncthreads();
    }

    // 4. update and stop-test partials
    const bool check = ((k + 1) % P.check_every == 0) || (k + 1 == P.k_end);
    CheckAcc acc;
    if (REG) {
      // A warp with a second row somewhere computes both rows' arithmetic first (no branch
      // between them, so they interleave), then the stop-test terms; a warp without one skips
      // it (warp-uniform).  A row past the end reads no sum, adds no terms and stores nothing.
      const bool in0 = tid < nr, in1 = tid + kThreads < nr;
      RowStep s0;
      if (__any_sync(0xffffffffu, in1)) {
        s0 = update_core(ry[0], rv[0], in0 ? S.sum[tid] : 0.0f, gam);
        const RowStep s1 = update_core(ry[1], rv[1], in1 ? S.sum[tid + kThreads] : 0.0f, gam);
        if (check && in1) check_terms(s1, ry[1], rv[1], rx[1], rw[1], th_lo, th_hi, acc);
        hits += in1 && !s1.ok ? 1ull : 0ull;
        ry[1] = s1.yn;
        rx[1] = s1.xn.hi;
        if (in1) {
          s_all[tid + kThreads] = ry[1].hi;
          if (!PUSH) yout[rb + tid + kThreads] = ry[1].hi;
        }
      } else {
        s0 = update_core(ry[0], rv[0], in0 ? S.sum[tid] : 0.0f, gam);
      }
      if (check && in0) check_terms(s0, ry[0], rv[0], rx[0], rw[0], th_lo, th_hi, acc);
      hits += in0 && !s0.ok ? 1ull : 0ull;
      ry[0] = s0.yn;
      rx[0] = s0.xn.hi;
      if (in0) {
        s_all[tid] = ry[0].hi;
        if (!PUSH) yout[rb + tid] = ry[0].hi;
      }
    } else {
      update_rows(S, nr, rb, P.w, PUSH ? nullptr : yout, gam, check, th_lo, th_hi, hits, acc);
    }
    gamma_store(gnext, T);  // visible to every thread after the next __syncthreads
    if (check && P.iterflag) write_check_partial(P, acc, slot, T);
    // 5. the new own states into the other CTAs' inboxes
    if (PUSH) {
      __syncthreads();
      push_states(piece, H.npiece, ssrc, s_all, inbox_out);
    }
    // 6. synchronisation and the stop decision (grid mode: at a check, fused into the barrier)
    if (P.iterflag)
      stop = publish_and_stop(P, fail, slot, check, gam, k, T);
    else if (check)
      stop = check_barrier(P, PUSH, fail, nbar, nchk, gam, k, acc, T);
    else
      stop = barrier_and_stop(P, PUSH, fail, nbar, slot, false, gam, k, T);
    synced = check;
    if (stop == 2) break;
    parity ^= 1;
    if (stop) {
      ++k;
      break;
    }
  }
  if (stop == 2) {
    // timeout: the status word says so.  A copy that this CTA started may still be in flight
    // into shared memory: wait for it (bounded) before the CTA exits; leave the state as is.
    if (PUSH && fail && H.lx > 0) mbar_wait(&s_bar, mphase ^ 1u, P.spin_limit);
    return;
  }
  float* yfin = parity ? P.y1 : P.y0;
  if (REG) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * kThreads;
      if (i < nr) {
        S.x[i] = rx[j];
        S.yl[i] = ry[j].lo;
        yfin[rb + i] = ry[j].hi;
      }
    }
    __syncthreads();
  } else {
    for (int i = tid; i < nr; i += blockDim.x) yfin[rb + i] = S.yh[i];
  }
  finish_run(P, S, rb, nr, hits, k, parity, T);
}

// ------------------------------------------------------------------------------------------
// host: the packed per-CTA blocks and the inboxes

static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Bank-conflict-free SELL columns.  In a slice, lane l's row has its entries (local ids, bank
// = id mod 32) and column c of the slice is one gather instruction over the 32 lanes.  The
// entries form a bipartite multigraph lanes x banks; colouring its edges with W colours so
// that no two edges at a lane or at a bank share a colour puts every lane's entries in
// distinct columns and every column's entries in distinct banks.  W colours suffice when W >=
// every lane's degree and every bank's load (Konig's edge-colouring theorem).  Alternating-path
// method: for an edge (l, b) take a colour a free at l and a
// colour c free at b; if a is also free at b use it, else swap a and c along the path from b
// whose edges alternate a, c, a, ... -- that frees a at b and cannot reach l, which has no
// a-edge.  lid[l] lists lane l's ids; the result col[l][k] is the column of lid[l][k].
struct ColorScratch {
  std::vector<int> at_l, at_b;           // [vertex * W + colour] -> edge, or -1 (built on demand)
  std::vector<uint64_t> used_l, used_b;  // the colours in use as bit sets: [vertex * nw + colour / 64]
  std::vector<int> elane, ebank, ecol, path;
};

// Most edges find a colour free at both ends; the edge tables the alternating paths walk are
// built only when the first edge of a slice does not.
static void color_slice(int W, const std::vector<uint16_t>* lid, std::vector<int>* col, ColorScratch& cs) {
  const int nw = (W + 63) >> 6;
  int E = 0;
  for (int l = 0; l < 32; ++l) E += (int)lid[l].size();
  std::vector<int>& at_l = cs.at_l;
  std::vector<int>& at_b = cs.at_b;
  std::vector<uint64_t>& ul = cs.used_l;
  std::vector<uint64_t>& ub = cs.used_b;
  int* elane = (cs.elane.resize(E), cs.elane.data());
  int* ebank = (cs.ebank.resize(E), cs.ebank.data());
  int* ecol = (cs.ecol.resize(E), cs.ecol.data());
  ul.assign(32 * (size_t)nw, 0);
  ub.assign(32 * (size_t)nw, 0);
  bool tables = false;
  // the lowest colour free at a vertex (one exists below W: its edges so far are fewer than W)
  auto lowest_free = [nw](const uint64_t* u) {
    int w = 0;
    while (w + 1 < nw && ~u[w] == 0) ++w;
    return w * 64 + __builtin_ctzll(~u[w]);
  };
  auto put = [&](int f, int x) {  // edge f takes colour x
    ecol[f] = x;
    ul[elane[f] * nw + (x >> 6)] |= 1ull << (x & 63);
    ub[ebank[f] * nw + (x >> 6)] |= 1ull << (x & 63);
    if (tables) {
      at_l[elane[f] * W + x] = f;
      at_b[ebank[f] * W + x] = f;
    }
  };
  auto take = [&](int f) {  // edge f gives up its colour (the tables are built)
    const int x = ecol[f];
    at_l[elane[f] * W + x] = -1;
    at_b[ebank[f] * W + x] = -1;
    ul[elane[f] * nw + (x >> 6)] &= ~(1ull << (x & 63));
    ub[ebank[f] * nw + (x >> 6)] &= ~(1ull << (x & 63));
  };
  int e = 0;
  for (int l = 0; l < 32; ++l) {
    for (size_t k = 0; k < lid[l].size(); ++k, ++e) {
      const int b = lid[l][k] & 31;
      elane[e] = l;
      ebank[e] = b;
      ecol[e] = -1;
      // the lowest colour free at both ends when there is one below W
      int a = -1;
      for (int w = 0; w < nw && a < 0; ++w) {
        const uint64_t both = ~(ul[(size_t)l * nw + w] | ub[(size_t)b * nw + w]);
        if (both) a = w * 64 + __builtin_ctzll(both);
      }
      if (a >= W) a = -1;
      if (a < 0) {
        // a free at l, c free at b: swap a and c along the a/c path from b
        if (!tables) {
          at_l.assign(32 * (size_t)W, -1);
          at_b.assign(32 * (size_t)W, -1);
          for (int f = 0; f < e; ++f) {
            at_l[elane[f] * W + ecol[f]] = f;
            at_b[ebank[f] * W + ecol[f]] = f;
          }
          tables = true;
        }
        a = lowest_free(&ul[(size_t)l * nw]);
        const int c = lowest_free(&ub[(size_t)b * nw]);
        std::vector<int>& path = cs.path;
        path.clear();
        int v = b, cur = a;
        bool bank_side = true;
        for (;;) {
          const int f = bank_side ? at_b[v * W + cur] : at_l[v * W + cur];
          if (f < 0) break;
          path.push_back(f);
          v = bank_side ? elane[f] : ebank[f];
          bank_side = !bank_side;
          cur = cur == a ? c : a;
        }
        for (int f : path) take(f);
        for (int f : path) put(f, ecol[f] == a ? c : a);
      }
      put(e, a);
    }
  }
  e = 0;
  for (int l = 0; l < 32; ++l) {
    col[l].resize(lid[l].size());
    for (size_t k = 0; k < lid[l].size(); ++k) col[l][k] = ecol[e++];
  }
}

// A CTA's halo is "dense" when it averages at least this many values per 32-byte sector:
// then the pull exchange reads few sectors and wins; below it the push exchange does.
static constexpr double kPullDensity = 4.0;

// Builds the blocks for the partition `part`, for the exchange `want` (GN_GATHER_HALO: by
// the halo density; GN_GATHER_HALO_PULL / _PUSH: that one).  Sets *fits = false (and builds
// nothing on the device) when a CTA's working set does not fit shared memory or 16-bit local
// ids; with the automatic choice the other exchange is tried before giving up.  The per-CTA
// work runs on the host threads, a CTA at a time (parallel_items); every CTA's output is its own.
static gn_status build_halo_blocks(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                                   const std::vector<int32_t>& part, const std::vector<std::vector<int32_t>>& ext,
                                   const std::vector<int64_t>& inbox_off, bool push, size_t smem_limit, bool* fits);

gn_status build_halo(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                     const std::vector<int32_t>& part, size_t smem_limit, int want, bool* fits) {
  *fits = false;
  const int nb = (int)part.size() - 1;
  const int n = g->n;

  // halos: each CTA's distinct external neighbours in increasing id order, from a bitmap of
  // the vertex range (a mark per entry, then a scan of the marked words), and the number of
  // 32-byte sectors of the state vector they touch
  std::vector<std::vector<int32_t>> ext(nb);
  std::vector<int64_t> sectors_of(nb, 0);
  std::vector<std::vector<uint64_t>> bitmaps(host_threads());  // per host thread, kept all-zero
  parallel_items(nb, [&](int b, int t) {
    std::vector<uint64_t>& bits = bitmaps[t];
    if (bits.empty()) bits.assign((size_t)n / 64 + 1, 0);
    {
      const int rb = part[b], re = part[b + 1];
      int wlo = INT32_MAX, whi = -1;
      for (int64_t e = rp[rb]; e < rp[re]; ++e) {
        const int j = ci[e];
        if (j >= rb && j < re) continue;
        bits[j >> 6] |= 1ull << (j & 63);
        wlo = std::min(wlo, j >> 6);
        whi = std::max(whi, j >> 6);
      }
      std::vector<int32_t>& xb = ext[b];
      int64_t sec = 0, last = -1;
      for (int wd = wlo; wd <= whi; ++wd) {
        uint64_t m = bits[wd];
        bits[wd] = 0;
        while (m) {
          const int j = wd * 64 + __builtin_ctzll(m);
          m &= m - 1;
          xb.push_back(j);
          sec += (j / 8 != last);
          last = j / 8;
        }
      }
      sectors_of[b] = sec;
    }
  });
  std::vector<int64_t> inbox_off(nb + 1, 0);
  int64_t vals = 0, sectors = 0;
  for (int b = 0; b < nb; ++b) {
    inbox_off[b + 1] = inbox_off[b] + (int64_t)((ext[b].size() + 3) & ~(size_t)3);
    vals += (int64_t)ext[b].size();
    sectors += sectors_of[b];
  }
  // the exchange: forced, or by the density of the halos in memory
  bool push = want == GN_GATHER_HALO_PUSH ||
              (want == GN_GATHER_HALO && (double)vals < kPullDensity * (double)std::max<int64_t>(sectors, 1));
  if (push && inbox_off[nb] > (int64_t)INT32_MAX) {  // inbox slots do not fit 32 bits
    if (want == GN_GATHER_HALO_PUSH) return GN_OK;
    push = false;
  }
  for (int attempt = 0; attempt < 2; ++attempt, push = !push) {
    if (attempt == 1 && want != GN_GATHER_HALO) break;
    gn_status st = build_halo_blocks(g, rp, ci, part, ext, inbox_off, push, smem_limit, fits);
    if (st != GN_OK || *fits) return st;
  }
  return GN_OK;
}

// The blocks for one exchange (see build_halo).
static gn_status build_halo_blocks(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                                   const std::vector<int32_t>& part, const std::vector<std::vector<int32_t>>& ext,
                                   const std::vector<int64_t>& inbox_off, bool push, size_t smem_limit, bool* fits) {
  *fits = false;
  const int nb = (int)part.size() - 1;
  const int n = g->n;
  int max_rows = 0;
  for (int b = 0; b < nb; ++b) max_rows = std::max(max_rows, part[b + 1] - part[b]);
  const int R = (max_rows + 3) & ~3;
  auto owner = [&](int j) { return (int)(std::upper_bound(part.begin(), part.end(), j) - part.begin()) - 1; };

  // send lists: for each owner o, the (inbox slot, own row) pairs in slot order.  The slots of
  // consumer c come before those of c + 1, and within c's halo (sorted by id) the vertices of
  // o are one run, found by binary search.
  std::vector<std::vector<std::pair<int32_t, int32_t>>> sends(nb);
  if (push) {
    parallel_items(nb, [&](int o, int) {
      {
        for (int c = 0; c < nb; ++c) {
          const std::vector<int32_t>& xc = ext[c];
          const size_t t0 = std::lower_bound(xc.begin(), xc.end(), part[o]) - xc.begin();
          const size_t t1 = std::lower_bound(xc.begin() + t0, xc.end(), part[o + 1]) - xc.begin();
          for (size_t t = t0; t < t1; ++t)
            sends[o].push_back({(int32_t)(inbox_off[c] + (int64_t)t), xc[t] - part[o]});
        }
      }
    });
  }

  // pass 1, per CTA: rows into interior / boundary / heavy, slices, chunks, send pieces and
  // the block layout
  std::vector<std::vector<unsigned char>> blocks(nb);
  parallel_items(nb, [&](int b, int) {
    {
      const int rb = part[b], re = part[b + 1], nr = re - rb;
      const std::vector<int32_t>& xb = ext[b];
      // the CTAs owning the halo (xb is sorted, the partition is contiguous)
      std::vector<int32_t> dep;
      for (int j : xb) {
        const int o = owner(j);
        if (dep.empty() || dep.back() != o) dep.push_back(o);
      }
      std::vector<int> light_int, light_bnd, heavy;
      for (int r = 0; r < nr; ++r) {
        const int64_t a = rp[rb + r], c = rp[rb + r + 1];
        if (c - a > kHeavyHalo) {
          heavy.push_back(r);
          continue;
        }
        bool bnd = false;
        for (int64_t e = a; e < c && !bnd; ++e) bnd = (ci[e] < rb || ci[e] >= re);
        (bnd ? light_bnd : light_int).push_back(r);
      }
      auto by_deg = [&](int x, int y) {
        const int dx = rp[rb + x + 1] - rp[rb + x], dy = rp[rb + y + 1] - rp[rb + y];
        return dx != dy ? dx > dy : x < y;
      };
      std::sort(light_int.begin(), light_int.end(), by_deg);
      std::sort(light_bnd.begin(), light_bnd.end(), by_deg);
      // interior-only slices first; the rest (the interior tail + boundary rows) after
      const int ns_int = (int)light_int.size() / 32;
      std::vector<int> order(light_int.begin(), light_int.end());
      order.insert(order.end(), light_bnd.begin(), light_bnd.end());
      const int ns = ((int)order.size() + 31) / 32;
      HaloHeader H;
      memset(&H, 0, sizeof H);
      H.ns_int = ns_int;
      H.ns = ns;
      H.nheavy = (int)heavy.size();
      H.lx = (int)xb.size();
      H.ndep = (int)dep.size();
      H.inbox_off = (int)inbox_off[b];
      std::vector<int2> meta(ns);
      std::vector<short> srow((size_t)ns * 32, (short)-1);
      int sell_len = 0;
      // slice width: the longest row (widening to the busiest bank's load, which would make
      // every gather conflict-free, measured slower: the extra columns cost more than the
      // conflicts they remove)
      for (int s = 0; s < ns; ++s) {
        int wmax = 0;
        for (int l = 0; l < 32; ++l) {
          const size_t q = (size_t)s * 32 + l;
          if (q < order.size()) {
            const int r = order[q];
            srow[q] = (short)r;
            wmax = std::max(wmax, (int)(rp[rb + r + 1] - rp[rb + r]));
          }
        }
        wmax = (wmax + 3) & ~3;
        meta[s] = make_int2(sell_len, wmax);
        sell_len += wmax * 32;
      }
      // heavy rows: (row, first chunk, chunks); chunks: (entry offset into hl, count)
      int heavy_len = 0;
      std::vector<int> hmeta, hchunk;
      for (int r : heavy) {
        const int d = rp[rb + r + 1] - rp[rb + r];
        hmeta.push_back(r);
        hmeta.push_back((int)hchunk.size() / 2);
        hmeta.push_back((d + kHeavyChunk - 1) / kHeavyChunk);
        for (int a = 0; a < d; a += kHeavyChunk) {
          hchunk.push_back(heavy_len + a);
          hchunk.push_back(std::min(kHeavyChunk, d - a));
        }
        heavy_len += d;
      }
      H.sell_len = sell_len;
      H.heavy_len = heavy_len;
      H.nchunk = (int)hchunk.size() / 2;
      // send pieces: runs of consecutive inbox slots, at most kSendPiece long
      const std::vector<std::pair<int32_t, int32_t>>& sd = sends[b];
      std::vector<int4> pieces;
      std::vector<uint16_t> src(sd.size());
      for (size_t e = 0; e < sd.size(); ++e) {
        src[e] = (uint16_t)sd[e].second;
        if (pieces.empty() || pieces.back().y == kSendPiece || sd[e].first != pieces.back().x + pieces.back().y)
          pieces.push_back(make_int4(sd[e].first, 0, (int)e, 0));
        ++pieces.back().y;
      }
      H.npiece = (int)pieces.size();
      size_t off = align16(sizeof(HaloHeader));
      H.off_meta = (int)off;
      off = align16(off + sizeof(int2) * ns);
      H.off_srow = (int)off;
      off = align16(off + sizeof(short) * 32 * (size_t)ns);
      H.off_sell = (int)off;
      off = align16(off + 2 * (size_t)sell_len);
      H.off_hmeta = (int)off;
      off = align16(off + 4 * hmeta.size());
      H.off_hl = (int)off;
      off = align16(off + 2 * (size_t)heavy_len);
      H.off_dep = (int)off;
      off = align16(off + 4 * dep.size());
      H.off_hchunk = (int)off;
      off = align16(off + 4 * hchunk.size());
      H.off_hpart = (int)off;
      off = align16(off + 4 * (size_t)H.nchunk);
      H.off_piece = (int)off;
      off = align16(off + sizeof(int4) * pieces.size());
      H.off_src = (int)off;
      off = align16(off + 2 * src.size());
      H.off_x = (int)off;
      if (!push) off = align16(off + 4 * xb.size());
      H.bytes = (int)off;
      std::vector<unsigned char>& B = blocks[b];
      B.assign(off, 0);
      memcpy(B.data(), &H, sizeof H);
      if (ns) memcpy(B.data() + H.off_meta, meta.data(), sizeof(int2) * ns);
      if (ns) memcpy(B.data() + H.off_srow, srow.data(), sizeof(short) * 32 * (size_t)ns);
      if (!hmeta.empty()) memcpy(B.data() + H.off_hmeta, hmeta.data(), 4 * hmeta.size());
      if (!dep.empty()) memcpy(B.data() + H.off_dep, dep.data(), 4 * dep.size());
      if (!hchunk.empty()) memcpy(B.data() + H.off_hchunk, hchunk.data(), 4 * hchunk.size());
      if (!pieces.empty()) memcpy(B.data() + H.off_piece, pieces.data(), sizeof(int4) * pieces.size());
      if (!src.empty()) memcpy(B.data() + H.off_src, src.data(), 2 * src.size());
      if (!push && !xb.empty()) memcpy(B.data() + H.off_x, xb.data(), 4 * xb.size());
    }
  });
  int lx_max = 0;
  size_t blk_max = 0;
  for (int b = 0; b < nb; ++b) {
    lx_max = std::max(lx_max, (int)ext[b].size());
    blk_max = std::max(blk_max, blocks[b].size());
  }
  const int Lp = (lx_max + 3) & ~3;
  const int zero_id = R + Lp;  // 32 zero slots from here, one per bank
  const size_t floats = (size_t)6 * R + Lp + 32;
  const size_t smem = 4 * floats + blk_max;
  if (zero_id + 31 > 65535 || smem > smem_limit || R > 32767) return GN_OK;  // does not fit

  // pass 2, per CTA: the 16-bit local ids (own row r -> r, external halo t -> R + t,
  // padding -> the zero slot)
  struct EncodeScratch {
    std::unique_ptr<int32_t[]> extpos;  // halo slot of each external id (set before it is read)
    std::vector<uint16_t> lids[32];
    std::vector<int> cols[32];
    ColorScratch cs;
    std::vector<int> occ;
    std::vector<uint16_t> bucket[32];
  };
  std::vector<EncodeScratch> scratch(host_threads());
  parallel_items(nb, [&](int b, int t) {
    EncodeScratch& X = scratch[t];
    if (!X.extpos) X.extpos.reset(new int32_t[std::max(n, 1)]);
    int32_t* extpos = X.extpos.get();
    std::vector<uint16_t>* lids = X.lids;
    std::vector<int>* cols = X.cols;
    ColorScratch& cs = X.cs;
    std::vector<int>& occ = X.occ;
    std::vector<uint16_t>* bucket = X.bucket;
    {
      const int rb = part[b], re = part[b + 1];
      std::vector<unsigned char>& B = blocks[b];
      HaloHeader* H = reinterpret_cast<HaloHeader*>(B.data());
      H->zero_id = zero_id;
      for (size_t t = 0; t < ext[b].size(); ++t) extpos[ext[b][t]] = (int32_t)t;
      auto lid = [&](int j) -> uint16_t {
        return (uint16_t)((j >= rb && j < re) ? (j - rb) : (R + extpos[j]));
      };
      const int2* meta = reinterpret_cast<const int2*>(B.data() + H->off_meta);
      const short* srow = reinterpret_cast<const short*>(B.data() + H->off_srow);
      uint16_t* sell = reinterpret_cast<uint16_t*>(B.data() + H->off_sell);
      // Every lane's row may list its entries in any order: colour the slice (color_slice) so
      // that each column's real entries lie in distinct banks, then pad each lane's empty
      // columns with the zero slot of a bank no real entry of that column uses (all padding of
      // a column reads that one address: a broadcast).
      for (int s = 0; s < H->ns; ++s) {
        const int W = meta[s].y;
        for (int l = 0; l < 32; ++l) {
          const int r = srow[s * 32 + l];
          lids[l].clear();
          if (r >= 0)
            for (int64_t e = rp[rb + r]; e < rp[rb + r + 1]; ++e) lids[l].push_back(lid(ci[e]));
        }
        // colours for the slice's busiest bank; when that is more than the slice's width, the
        // colours past the width fold into each lane's free columns, least-used bank first
        // (only those gathers can conflict)
        int Wc = W, load[32] = {0};
        for (int l = 0; l < 32; ++l)
          for (uint16_t id : lids[l]) ++load[id & 31];
        for (int t = 0; t < 32; ++t) Wc = std::max(Wc, load[t]);
        color_slice(Wc, lids, cols, cs);
        occ.assign(32 * (size_t)W, 0);  // occ[bank * W + column]
        for (int l = 0; l < 32; ++l)
          for (size_t t = 0; t < lids[l].size(); ++t)
            if (cols[l][t] < W) ++occ[(lids[l][t] & 31) * W + cols[l][t]];
        if (Wc > W) {
          for (int l = 0; l < 32; ++l) {
            uint64_t used = 0;
            for (size_t t = 0; t < lids[l].size(); ++t)
              if (cols[l][t] < W) used |= 1ull << cols[l][t];
            for (size_t t = 0; t < lids[l].size(); ++t) {
              if (cols[l][t] < W) continue;
              const int bk = lids[l][t] & 31;
              int best = -1;
              for (int k = 0; k < W; ++k)
                if (!(used >> k & 1ull) && (best < 0 || occ[bk * W + k] < occ[bk * W + best])) best = k;
              cols[l][t] = best;
              used |= 1ull << best;
              ++occ[bk * W + best];
            }
          }
        }
        for (int k = 0; k < W; ++k) {
          int zb = 0;  // the bank least used by column k's real entries (unused when one exists)
          for (int t = 1; t < 32; ++t)
            if (occ[t * W + k] < occ[zb * W + k]) zb = t;
          const uint16_t zero = (uint16_t)(zero_id + ((zb - zero_id) & 31));
          for (int l = 0; l < 32; ++l) sell[meta[s].x + (k >> 2) * 128 + l * 4 + (k & 3)] = zero;
        }
        for (int l = 0; l < 32; ++l)
          for (size_t t = 0; t < lids[l].size(); ++t) {
            const int k = cols[l][t];
            sell[meta[s].x + (k >> 2) * 128 + l * 4 + (k & 3)] = lids[l][t];
          }
      }
      const int* hm = reinterpret_cast<const int*>(B.data() + H->off_hmeta);
      const int* hc = reinterpret_cast<const int*>(B.data() + H->off_hchunk);
      uint16_t* hl = reinterpret_cast<uint16_t*>(B.data() + H->off_hl);
      // heavy rows: entries dealt round-robin over the banks, so each group of 32 consecutive
      // entries (one gather instruction of sum_chunk) spreads over the banks
      for (int h = 0; h < H->nheavy; ++h) {
        const int r = hm[3 * h], o = hc[2 * hm[3 * h + 1]];  // the row's entries start at its first chunk
        const int d = rp[rb + r + 1] - rp[rb + r];
        size_t most = 0;
        for (int t = 0; t < 32; ++t) bucket[t].clear();
        for (int k = 0; k < d; ++k) {
          const uint16_t id = lid(ci[rp[rb + r] + k]);
          bucket[id & 31].push_back(id);
        }
        for (int t = 0; t < 32; ++t) most = std::max(most, bucket[t].size());
        int k = 0;
        for (size_t j = 0; j < most; ++j)
          for (int t = 0; t < 32; ++t)
            if (j < bucket[t].size()) hl[o + k++] = bucket[t][j];
      }
    }
  });
  std::vector<int64_t> hoff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) hoff[b + 1] = hoff[b] + (int64_t)blocks[b].size();
  std::vector<unsigned char> blob((size_t)std::max<int64_t>(hoff[nb], 16));
  parallel_for(nb, 8, [&](int lo, int hi, int) {
    for (int b = lo; b < hi; ++b) memcpy(blob.data() + hoff[b], blocks[b].data(), blocks[b].size());
  });
  GN_CUDA(cudaMalloc(&g->d_hoff, sizeof(int64_t) * (nb + 1)));
  GN_CUDA(cudaMalloc(&g->d_hblob, blob.size()));
  if (push) {
    g->inbox_len = std::max<int64_t>(inbox_off[nb], 4);
    GN_CUDA(cudaMalloc(&g->d_inbox, sizeof(float) * 2 * (size_t)g->inbox_len));
    GN_CUDA(cudaMemsetAsync(g->d_inbox, 0, sizeof(float) * 2 * (size_t)g->inbox_len, g->stream));
  }
  g->halo_push = push;
  GN_CUDA(cudaMemcpyAsync(g->d_hoff, hoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(g->d_hblob, blob.data(), blob.size(), cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  g->halo_pad = Lp;
  g->rows_pad_halo = R;
  g->smem_bytes = smem;
  *fits = true;
  return GN_OK;
}

const void* halo_kernel(int rows_pad, bool push) {
  if (push) return rows_pad <= 2 * kThreads ? (const void*)k_gn_halo<true, true> : (const void*)k_gn_halo<false, true>;
  return rows_pad <= 2 * kThreads ? (const void*)k_gn_halo<true, false> : (const void*)k_gn_halo<false, false>;
}

}  // namespace gn
