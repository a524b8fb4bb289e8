// gn_halo.cu -- the halo gather mode of the persistent WRGN kernel.
//
// Each CTA owns a contiguous range of rows for the whole run and keeps everything it needs
// in shared memory:
//   s_all  = [ own weighted states y_i (hi parts) | external halo values | 32 zeros ]
//   a packed per-CTA block (gn_halo.cuh, built once on the host by gn_halo_build.cu): the
//   light rows in SELL-32 slices (32 rows per slice, a lane per row, 16-bit local ids into
//   s_all packed four per lane in 8-byte words, rows sorted interior-first then by degree;
//   each column is one gather instruction and touches 32 distinct banks, see color_slice),
//   the heavy rows cut into chunks of at most 256 entries (a warp per chunk; a row's chunk
//   sums are added in chunk order, so the result does not depend on which warp took which
//   chunk) and the CTA's send list.
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

#include "gn_halo.cuh"
#include "gn_iter_common.cuh"

namespace gn {

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

// tagged exchange: the tag bit of a halo value (its sign; every weighted state is >= +0), the
// halo slots per thread loaded before the interior sums, and per batch after them
constexpr unsigned kTagBit = 0x80000000u;
constexpr int kTagPre = 2;
constexpr int kTagBatch = 8;
// push: the inbox is contiguous, so a thread reads four consecutive slots with one 16-byte
// load (four 4-byte accesses, each with its own tag), kTagGroups such groups at a time (the
// first ones issued before the interior sums)
constexpr int kTagGroups = 4;


// push: the send list, own states (s_all) into the other CTAs' inboxes, a warp per piece of
// at most 128 slots, lane j storing slots 4j .. 4j + 3 of the piece with one 16-byte store
// (pieces start at multiples of 4 slots); the four ids come in one 8-byte load, and the
// builder placed the values so that each of the four gathers reads distinct banks where it
// could.  TAG: each value goes out with tag bit `tag` in its sign (four 4-byte relaxed
// accesses in one vector store).
template <bool TAG>
__device__ __forceinline__ void push_states(const int4* __restrict__ piece, int npiece,
                                            const uint16_t* __restrict__ src, const float* __restrict__ s_all,
                                            float* __restrict__ inbox, unsigned tag = 0u) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int q = warp; q < npiece; q += nwarps) {
    const int4 pc = piece[q];
    if (4 * lane < pc.y) {
      const uint2 ids = *reinterpret_cast<const uint2*>(src + pc.z + 4 * lane);
      const float a = s_all[ids.x & 0xffffu], b = s_all[ids.x >> 16], c = s_all[ids.y & 0xffffu],
                  d = s_all[ids.y >> 16];
      if (TAG) {
        asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(
                         reinterpret_cast<unsigned*>(inbox) + pc.x + 4 * lane),
                     "r"((__float_as_uint(a) & ~kTagBit) | tag), "r"((__float_as_uint(b) & ~kTagBit) | tag),
                     "r"((__float_as_uint(c) & ~kTagBit) | tag), "r"((__float_as_uint(d) & ~kTagBit) | tag)
                     : "memory");
      } else {
        *reinterpret_cast<float4*>(inbox + pc.x + 4 * lane) = make_float4(a, b, c, d);
      }
    }
  }
}

// tagged exchange: a halo slot's value once its tag bit is `want`, polling again until then;
// bounded like the barriers (a limit, or another CTA's reported failure, sets `fail`); with
// `fail` already set it returns at once
__device__ __forceinline__ unsigned poll_tag(const unsigned* p, unsigned v, unsigned want, const IterParams& P,
                                             bool& fail) {
  long long spins = 0;
  while (((v ^ want) & kTagBit) && !fail) {
    ++spins;
    if ((spins & 255) == 0 && dev::ld_relaxed_int(P.status) != 0) {
      fail = true;
    } else if (spins > P.spin_limit) {
      atomicOr(P.status, DEV_TIMEOUT);
      fail = true;
    } else {
      v = dev::ld_relaxed(p);
    }
  }
  return v;
}

__device__ __forceinline__ uint4 ld_relaxed_v4(const uint4* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

// push, tagged: whether the slots 4q .. 4q + 3 below lx all carry tag `want`
__device__ __forceinline__ bool ready4(uint4 v, int q, int lx, unsigned want) {
  const int t = 4 * q;
  const unsigned m = ((v.x ^ want) | (t + 1 < lx ? v.y ^ want : 0u) | (t + 2 < lx ? v.z ^ want : 0u) |
                      (t + 3 < lx ? v.w ^ want : 0u));
  return !(m & kTagBit);
}

// push, tagged: this thread's groups q = q0 + u * kThreads (u < kTagGroups) of four consecutive
// inbox slots, v[u] already loaded once.  Every round reloads all the groups that still hold
// a slot with another tag, together (one round trip per round), bounded like the barriers;
// then the values, tags cleared, into the halo.
__device__ __forceinline__ void land_tagged4(uint4 (&v)[kTagGroups], int q0, int lx, const uint4* __restrict__ src4,
                                             float* __restrict__ s_halo, unsigned want, const IterParams& P,
                                             bool& fail) {
  long long spins = 0;
  for (;;) {
    bool done = true;
#pragma unroll
    for (int u = 0; u < kTagGroups; ++u) {
      const int q = q0 + u * kThreads;
      if (4 * q < lx && !ready4(v[u], q, lx, want)) done = false;
    }
    if (done || fail) break;
    ++spins;
    if ((spins & 255) == 0 && dev::ld_relaxed_int(P.status) != 0) {
      fail = true;
      break;
    }
    if (spins > P.spin_limit) {
      atomicOr(P.status, DEV_TIMEOUT);
      fail = true;
      break;
    }
#pragma unroll
    for (int u = 0; u < kTagGroups; ++u) {
      const int q = q0 + u * kThreads;
      if (4 * q < lx && !ready4(v[u], q, lx, want)) v[u] = ld_relaxed_v4(src4 + q);
    }
  }
#pragma unroll
  for (int u = 0; u < kTagGroups; ++u) {
    const int q = q0 + u * kThreads, t = 4 * q;
    if (t + 3 < lx) {
      reinterpret_cast<float4*>(s_halo)[q] =
          make_float4(__uint_as_float(v[u].x & ~kTagBit), __uint_as_float(v[u].y & ~kTagBit),
                      __uint_as_float(v[u].z & ~kTagBit), __uint_as_float(v[u].w & ~kTagBit));
    } else if (t < lx) {
      s_halo[t] = __uint_as_float(v[u].x & ~kTagBit);
      if (t + 1 < lx) s_halo[t + 1] = __uint_as_float(v[u].y & ~kTagBit);
      if (t + 2 < lx) s_halo[t + 2] = __uint_as_float(v[u].z & ~kTagBit);
    }
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
// TAG: the tagged exchange (no grid barrier between checks), else the barrier or the flags.
template <bool REG, bool PUSH, bool TAG>
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
  Own ro[2];
  dev::f2 rv[2];
  float rw[2];
  if (REG) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * kThreads;
      const bool in = i < nr;
      // a row past the CTA's end is a fixed point y = x = 1 (never a safe division)
      ro[j] = in ? own_load(P.y0[rb + i], P.ylo[rb + i], P.x[rb + i], P.yexp[rb + i]) : Own{1.0f, 0.0f, 1.0f};
      rv[j] = in ? dev::f2{P.v[rb + i], P.vlo[rb + i]} : dev::f2{1.0f, 0.0f};
      rw[j] = in ? P.w[rb + i] : 0.0f;
      if (in) S.yh[i] = ro[j].pub;
    }
  } else {
    for (int i = tid; i < nr; i += blockDim.x) {
      S.vh[i] = P.v[rb + i];
      S.vl[i] = P.vlo[rb + i];
      const Own o = own_load(P.y0[rb + i], P.ylo[rb + i], P.x[rb + i], P.yexp[rb + i]);
      S.yh[i] = o.pub;
      S.yl[i] = o.aux;
      S.x[i] = o.xs;
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

  // tagged exchange: three buffers of inbox_len slots (push: the inboxes; pull: one slot per
  // vertex); iteration r reads buffer r % 3, whose values carry tag bit (r / 3) % 2
  // (the buffers' base and length are re-read from the launch parameters where they are used,
  // which keeps them out of the registers)
#define TBUF reinterpret_cast<unsigned*>(P.inbox)
#define TLEN ((size_t)P.inbox_len)
  // tagged exchange state: the buffer index (bits 0..1) and the tag bit of this iteration
  unsigned tcode = P.bad_tag ? kTagBit : 0u;

  unsigned hits = 0;
  int parity = 0, slot = 0, stop = 0;
  unsigned nbar = 0;
  int nchk = 0;  // checks so far (grid mode: selects the check word)
  unsigned mphase = 0;  // parity of the mbarrier phase the next copy completes
  int k = P.k_start;

  // prologue: the starting states into inbox[0] (push), then every CTA's halo is complete.
  // Tagged: the starting states into buffer 0 with tag 0, and this CTA's slots of buffers 1 and
  // 2 marked with tag 1, which their first readers (iterations 1 and 2, tag 0) do not accept.
  if (TAG) {
    if (PUSH) {
      push_states<true>(piece, H.npiece, ssrc, s_all, P.inbox, 0u);
      push_states<true>(piece, H.npiece, ssrc, s_all, P.inbox + TLEN, kTagBit);
      push_states<true>(piece, H.npiece, ssrc, s_all, P.inbox + 2 * TLEN, kTagBit);
    } else {
      for (int i = tid; i < nr; i += blockDim.x) {
        const unsigned u = __float_as_uint(s_all[i]) & ~kTagBit;
        dev::st_relaxed_u32(TBUF + rb + i, u);
        dev::st_relaxed_u32(TBUF + TLEN + rb + i, u | kTagBit);
        dev::st_relaxed_u32(TBUF + 2 * TLEN + rb + i, u | kTagBit);
      }
    }
  } else if (PUSH) {
    push_states<false>(piece, H.npiece, ssrc, s_all, P.inbox);
  }
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
  int next_chk = (P.k_start / P.check_every + 1) * P.check_every;  // a check follows step next_chk - 1

  for (; stop != 2 && k < P.k_end; ++k) {
    const int r = k - P.k_start;
    const dev::f2 gam = {T.gh, T.gl};
    const float2 gnext = gamma_fetch(P, k + 1);
    const float* inbox_in = PUSH ? P.inbox + (size_t)(r & 1) * (size_t)P.inbox_len : nullptr;
    float* inbox_out = PUSH ? P.inbox + (size_t)((r + 1) & 1) * (size_t)P.inbox_len : nullptr;
    const float* __restrict__ yin = parity ? P.y1 : P.y0;  // pull
    float* __restrict__ yout = parity ? P.y0 : P.y1;
    const unsigned tbit = tcode & kTagBit;  // tagged: this iteration's tag,
    const unsigned ocode = (tcode & 3u) == 2u ? (tcode ^ kTagBit) & kTagBit : tcode + 1u;  // and r + 1's
    const unsigned obit = ocode & kTagBit;
    const unsigned* tin = TBUF + (size_t)(tcode & 3u) * TLEN;
    unsigned* tout = TBUF + (size_t)(ocode & 3u) * TLEN;

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
    // 1. the halo, asynchronously (tagged: each thread's first kTagPre slots, in flight during
    // the interior sums)
    unsigned pre[kTagPre];
    uint4 pre4[kTagGroups];
    if (TAG && PUSH) {
      const uint4* src4 = reinterpret_cast<const uint4*>(tin + H.inbox_off);
#pragma unroll
      for (int u = 0; u < kTagGroups; ++u) {
        const int q = tid + u * kThreads;
        pre4[u] = 4 * q < H.lx ? ld_relaxed_v4(src4 + q) : make_uint4(0u, 0u, 0u, 0u);
      }
    } else if (TAG) {
#pragma unroll
      for (int u = 0; u < kTagPre; ++u) {
        const int t = tid + u * kThreads;
        pre[u] = t < H.lx ? dev::ld_relaxed(tin + xlist[t]) : 0u;
      }
    } else if (PUSH) {
      if (tid == 0 && H.lx > 0 && !fail) bulk_fetch(s_halo, inbox_in + H.inbox_off, halo_bytes, &s_bar);
    } else {
      for (int t = tid; t < H.lx; t += blockDim.x) cp_async4(&s_halo[t], yin + xlist[t]);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    // 2. interior rows need only own values
    for (int s = warp; s < H.ns_int; s += nwarps) sum_slice(s, meta, srow, sell, s_all, S.sum);
    // 3. boundary rows and heavy chunks after the halo has landed.  Tagged: a slot whose tag is
    // not yet this iteration's is polled again; the slots past the first kTagPre per thread are
    // loaded kTagBatch at a time
    if (TAG && PUSH) {
      const uint4* src4 = reinterpret_cast<const uint4*>(tin + H.inbox_off);
      land_tagged4(pre4, tid, H.lx, src4, s_halo, tbit, P, fail);
      for (int q0 = tid + kTagGroups * kThreads; 4 * q0 < H.lx; q0 += kTagGroups * kThreads) {
#pragma unroll
        for (int u = 0; u < kTagGroups; ++u) {
          const int q = q0 + u * kThreads;
          pre4[u] = 4 * q < H.lx ? ld_relaxed_v4(src4 + q) : make_uint4(0u, 0u, 0u, 0u);
        }
        land_tagged4(pre4, q0, H.lx, src4, s_halo, tbit, P, fail);
      }
    } else if (TAG) {
#pragma unroll
      for (int u = 0; u < kTagPre; ++u) {
        const int t = tid + u * kThreads;
        if (t < H.lx) s_halo[t] = __uint_as_float(poll_tag(tin + xlist[t], pre[u], tbit, P, fail) & ~kTagBit);
      }
      for (int t0 = tid + kTagPre * kThreads; t0 < H.lx; t0 += kTagBatch * kThreads) {
        unsigned v[kTagBatch];
#pragma unroll
        for (int u = 0; u < kTagBatch; ++u) {
          const int t = t0 + u * kThreads;
          v[u] = t < H.lx ? dev::ld_relaxed(tin + xlist[t]) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kTagBatch; ++u) {
          const int t = t0 + u * kThreads;
          if (t < H.lx) s_halo[t] = __uint_as_float(poll_tag(tin + xlist[t], v[u], tbit, P, fail) & ~kTagBit);
        }
      }
    }
    if (TAG) {
      if (__syncthreads_or(fail)) {
        stop = 2;
        break;
      }
    } else if (PUSH) {
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
    if (!TAG) __syncthreads();
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
    const bool due = k + 1 == next_chk;
    const bool check = due || (k + 1 == P.k_end);
    if (due) next_chk += P.check_every;
    CheckAcc acc;
    if (REG) {
      // A warp with a second row somewhere computes both rows' arithmetic first (no branch
      // between them, so they interleave), then the stop-test terms; a warp without one skips
      // it (warp-uniform).  A row past the end reads no sum, adds no terms and stores nothing.
      const bool in0 = tid < nr, in1 = tid + kThreads < nr;
      RowStep s0;
      if (__any_sync(0xffffffffu, in1)) {
        s0 = update_core(ro[0], rv[0], in0 ? S.sum[tid] : 0.0f, gam);
        const RowStep s1 = update_core(ro[1], rv[1], in1 ? S.sum[tid + kThreads] : 0.0f, gam);
        if (check && in1) check_terms(s1, ro[1], rv[1], rw[1], th_lo, th_hi, acc);
        hits += in1 && !s1.ok ? 1u : 0u;
        ro[1] = s1.next;
        if (in1) {
          s_all[tid + kThreads] = ro[1].pub;
          if (!PUSH && TAG) dev::st_relaxed_u32(tout + rb + tid + kThreads, (__float_as_uint(ro[1].pub) & ~kTagBit) | obit);
          if (!PUSH && !TAG) yout[rb + tid + kThreads] = ro[1].pub;
        }
      } else {
        s0 = update_core(ro[0], rv[0], in0 ? S.sum[tid] : 0.0f, gam);
      }
      if (check && in0) check_terms(s0, ro[0], rv[0], rw[0], th_lo, th_hi, acc);
      hits += in0 && !s0.ok ? 1u : 0u;
      ro[0] = s0.next;
      if (in0) {
        s_all[tid] = ro[0].pub;
        if (!PUSH && TAG) dev::st_relaxed_u32(tout + rb + tid, (__float_as_uint(ro[0].pub) & ~kTagBit) | obit);
        if (!PUSH && !TAG) yout[rb + tid] = ro[0].pub;
      }
    } else {
      // one row at a time: interleaving two rows (update_rows) needs more than the 64 registers
      // a 1024-thread CTA allows next to this kernel's state and spills (4% slower on BA)
      for (int i = tid; i < nr; i += blockDim.x) {
        Own o = {S.yh[i], S.yl[i], S.x[i]};
        update_one(o, dev::f2{S.vh[i], S.vl[i]}, S.sum[i], gam, check, check ? P.w[rb + i] : 0.0f, th_lo, th_hi,
                   hits, acc);
        S.yh[i] = o.pub;
        S.yl[i] = o.aux;
        S.x[i] = o.xs;
        if (!PUSH && TAG) dev::st_relaxed_u32(tout + rb + i, (__float_as_uint(o.pub) & ~kTagBit) | obit);
        if (!PUSH && !TAG) yout[rb + i] = o.pub;
      }
    }
    gamma_store(gnext, T);  // visible to every thread after the next __syncthreads
    if (check && P.iterflag) write_check_partial(P, acc, slot, T);
    // 5. the new own states into the other CTAs' inboxes
    if (PUSH) {
      __syncthreads();
      if (TAG)
        push_states<true>(piece, H.npiece, ssrc, s_all, P.inbox + (size_t)(ocode & 3u) * TLEN, obit);
      else
        push_states<false>(piece, H.npiece, ssrc, s_all, inbox_out);
    }
    // 6. synchronisation and the stop decision (grid mode: at a check, fused into the barrier).
    // Tagged, between checks: only a bar.sync (pull: the own values of this update before the
    // next interior sums; push has one before its stores)
    if (P.iterflag) {
      stop = publish_and_stop(P, fail, slot, check, gam, k, T);
    } else if (check) {
      stop = check_barrier(P, PUSH || TAG, fail, nbar, nchk, gam, k, acc, T);
    } else if (TAG) {
      stop = 0;
      if (!PUSH) __syncthreads();
    } else {
      stop = barrier_and_stop(P, PUSH, fail, nbar, slot, false, gam, k, T);
    }
    synced = check;
    tcode = ocode;
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
    if (!TAG && PUSH && fail && H.lx > 0) mbar_wait(&s_bar, mphase ^ 1u, P.spin_limit);
    return;
  }
  float* yfin = parity ? P.y1 : P.y0;
  if (REG) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * kThreads;
      if (i < nr) {
        S.x[i] = ro[j].xs;
        S.yl[i] = ro[j].aux;
        S.vh[i] = rv[j].hi;  // own_x reads it
        yfin[rb + i] = ro[j].pub;
      }
    }
    __syncthreads();
  } else {
    for (int i = tid; i < nr; i += blockDim.x) yfin[rb + i] = S.yh[i];
  }
#undef TBUF
#undef TLEN
  finish_run(P, S, rb, nr, hits, k, parity, T);
}

const void* halo_kernel(int rows_pad, bool push, bool tagged) {
  const bool reg = rows_pad <= 2 * kThreads;
  if (tagged) {
    if (push) return reg ? (const void*)k_gn_halo<true, true, true> : (const void*)k_gn_halo<false, true, true>;
    return reg ? (const void*)k_gn_halo<true, false, true> : (const void*)k_gn_halo<false, false, true>;
  }
  if (push) return reg ? (const void*)k_gn_halo<true, true, false> : (const void*)k_gn_halo<false, true, false>;
  return reg ? (const void*)k_gn_halo<true, false, false> : (const void*)k_gn_halo<false, false, false>;
}

}  // namespace gn
