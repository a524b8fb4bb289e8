// gn_halo.cu -- the halo gather mode of the persistent WRGN kernel.
//
// Each CTA owns a contiguous range of rows for the whole run and keeps everything it needs
// in shared memory:
//   s_all  = [ own weighted states y_i (hi parts) | external halo values | one zero ]
//   a packed per-CTA block (built once on the host): the list of external neighbour ids,
//   the light rows in SELL-32 slices (32 rows per slice, a lane per row, 16-bit local ids
//   into s_all packed four per lane in 8-byte words, rows sorted interior-first then by
//   degree, each column's entries spread over the shared-memory banks) and the heavy rows
//   (a warp per row).
// One iteration:
//   1. cp.async copies of the external halo values y_j (written by other CTAs last iteration)
//   2. row sums of the interior slices (only own rows: no wait) while the copies fly
//   3. wait for the copies; row sums of the boundary slices and of the heavy rows
//   4. the update (gn_iter_common.cuh), the stop-test partials, the bounded grid barrier
// Only the distinct external neighbours of a CTA are read from L2 each iteration; every
// other read is shared memory.
#include <algorithm>
#include <cstring>
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
  int zero_id;     // local id of the zero slot (padding)
  int off_x;       // byte offsets of the sections from the block start
  int off_meta;
  int off_srow;
  int off_sell;
  int off_hmeta;
  int off_hl;
  int bytes;       // block size (multiple of 16)
  int pad0, pad1;
};

static constexpr int kHeavyHalo = 64;  // rows with more entries go warp-per-row

__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// SELL-32 slices [s0, s1): warp per slice, lane per row.  A slice's width is a multiple of 4
// and each lane's local ids come four at a time in one 8-byte word (layout [k/4][lane]).
__device__ __forceinline__ void sum_slices(int s0, int s1, const int2* __restrict__ meta,
                                           const short* __restrict__ srow,
                                           const uint16_t* __restrict__ sell,
                                           const float* __restrict__ s_all, float* __restrict__ s_sum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int s = s0 + warp; s < s1; s += nwarps) {
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
}

// REG: a CTA owns at most 2 * kThreads rows and each thread keeps its (at most two) rows'
// state in registers across iterations; only y (for the neighbour sums) goes to shared memory.
template <bool REG>
__global__ void __launch_bounds__(kThreads, 1) k_gn_halo(const IterParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TailShared T;
  const int R = P.rows_pad;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int b = blockIdx.x;
  const int rb = P.part[b], nr = P.part[b + 1] - rb;

  // a failed start-state validation (written before the launch) ends the run at once
  if (dev::ld_relaxed_int(P.status) != 0) return;

  float* s_all = reinterpret_cast<float*>(smem);
  const int nall = R + P.halo_pad + 4;
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
      ry[j] = in ? dev::f2{P.y0[rb + i], P.ylo[rb + i]} : dev::f2{0.0f, 0.0f};
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
  __syncthreads();
  const HaloHeader H = *reinterpret_cast<const HaloHeader*>(blk);
  const int* __restrict__ xlist = reinterpret_cast<const int*>(blk + H.off_x);
  const int2* __restrict__ meta = reinterpret_cast<const int2*>(blk + H.off_meta);
  const short* __restrict__ srow = reinterpret_cast<const short*>(blk + H.off_srow);
  const uint16_t* __restrict__ sell = reinterpret_cast<const uint16_t*>(blk + H.off_sell);
  const int* __restrict__ hmeta = reinterpret_cast<const int*>(blk + H.off_hmeta);
  const uint16_t* __restrict__ hl = reinterpret_cast<const uint16_t*>(blk + H.off_hl);
  if (tid == 0) s_all[H.zero_id] = 0.0f;
  set_gamma(P, P.k_start, T);
  float* s_halo = s_all + R;
  const float th_lo = (float)P.theta, th_hi = (float)(1.0 - P.theta);
  __syncthreads();

  unsigned long long hits = 0;
  int parity = 0, slot = 0, stop = 0;
  unsigned nbar = 0;
  int k = P.k_start;

  for (; k < P.k_end; ++k) {
    const double gam_d = T.gd;
    const dev::f2 gam = {T.gh, T.gl};
    const float2 gnext = gamma_fetch(P, k + 1);
    const float* __restrict__ yin = parity ? P.y1 : P.y0;
    float* __restrict__ yout = parity ? P.y0 : P.y1;

    // 1. external halo values, asynchronously
    for (int t = tid; t < H.lx; t += blockDim.x) cp_async4(&s_halo[t], yin + xlist[t]);
    cp_async_commit();
    // 2. interior rows need only own values
    sum_slices(0, H.ns_int, meta, srow, sell, s_all, S.sum);
    // 3. boundary rows and heavy rows after the halo has landed
    cp_async_wait_all();
    __syncthreads();
    sum_slices(H.ns_int, H.ns, meta, srow, sell, s_all, S.sum);
    for (int h = warp; h < H.nheavy; h += nwarps) {
      const int r = hmeta[3 * h], a = hmeta[3 * h + 1], c = a + hmeta[3 * h + 2];
      float acc = 0.0f;
      for (int e = a + lane; e < c; e += 32) acc += s_all[hl[e]];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) S.sum[r] = acc;
    }
    __syncthreads();

    // 4. update, stop-test partials, barrier, stop decision
    const bool check = ((k + 1) % P.check_every == 0) || (k + 1 == P.k_end);
    CheckAcc acc;
    if (REG) {
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int i = tid + j * kThreads;
        if (i < nr) {
          update_one(ry[j], rv[j], rx[j], S.sum[i], gam, check, rw[j], th_lo, th_hi, hits, acc);
          s_all[i] = ry[j].hi;
          yout[rb + i] = ry[j].hi;
        }
      }
    } else {
      update_rows(S, nr, rb, P.w, yout, gam, check, th_lo, th_hi, hits, acc);
    }
    gamma_store(gnext, T);  // visible to every thread after the barrier's __syncthreads
    if (check) write_check_partial(P, acc, slot, T);
    stop = barrier_and_stop(P, nbar, slot, check, gam_d, k, T);
    if (stop == 2) break;
    parity ^= 1;
    if (stop) {
      ++k;
      break;
    }
  }
  if (stop == 2) return;  // timeout: the status word says so; leave the state as is
  if (REG) {
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int i = tid + j * kThreads;
      if (i < nr) {
        S.x[i] = rx[j];
        S.yl[i] = ry[j].lo;
      }
    }
    __syncthreads();
  }
  finish_run(P, S, rb, nr, hits, k, parity, T);
}

// ------------------------------------------------------------------------------------------
// host: the packed per-CTA blocks

static size_t align16(size_t b) { return (b + 15) & ~(size_t)15; }

// Builds the blocks for the partition `part`.  Returns false (and builds nothing on the
// device) when a CTA's working set does not fit shared memory or 16-bit local ids.
gn_status build_halo(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                     const std::vector<int32_t>& part, size_t smem_limit, bool* fits) {
  *fits = false;
  const int nb = (int)part.size() - 1;
  const int n = g->n;
  int max_rows = 0;
  for (int b = 0; b < nb; ++b) max_rows = std::max(max_rows, part[b + 1] - part[b]);
  const int R = (max_rows + 3) & ~3;

  std::vector<std::vector<unsigned char>> blocks(nb);
  std::vector<int32_t> stamp(std::max(n, 1), -1), extpos(std::max(n, 1), 0);
  int lx_max = 0;
  size_t blk_max = 0;
  for (int b = 0; b < nb; ++b) {
    const int rb = part[b], re = part[b + 1], nr = re - rb;
    // external halo: distinct neighbours outside [rb, re), sorted
    std::vector<int32_t> ext;
    for (int64_t e = rp[rb]; e < rp[re]; ++e) {
      const int j = ci[e];
      if ((j < rb || j >= re) && stamp[j] != b) {
        stamp[j] = b;
        ext.push_back(j);
      }
    }
    std::sort(ext.begin(), ext.end());
    for (size_t t = 0; t < ext.size(); ++t) extpos[ext[t]] = (int32_t)t;
    lx_max = std::max(lx_max, (int)ext.size());
    blocks[b].clear();
    // the local ids need the final halo padding; gather rows first, encode after
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
    // store the structure as a plain vector of ints for encoding later
    HaloHeader H;
    memset(&H, 0, sizeof H);
    H.ns_int = ns_int;
    H.ns = ns;
    H.nheavy = (int)heavy.size();
    H.lx = (int)ext.size();
    std::vector<int2> meta(ns);
    std::vector<short> srow((size_t)ns * 32, (short)-1);
    int sell_len = 0;
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
    int heavy_len = 0;
    std::vector<int> hmeta;
    for (int r : heavy) {
      const int d = rp[rb + r + 1] - rp[rb + r];
      hmeta.push_back(r);
      hmeta.push_back(heavy_len);
      hmeta.push_back(d);
      heavy_len += d;
    }
    H.sell_len = sell_len;
    H.heavy_len = heavy_len;
    size_t off = align16(sizeof(HaloHeader));
    H.off_x = (int)off;
    off = align16(off + 4 * ext.size());
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
    H.bytes = (int)off;
    blk_max = std::max(blk_max, off);
    std::vector<unsigned char>& B = blocks[b];
    B.assign(off, 0);
    memcpy(B.data(), &H, sizeof H);
    if (!ext.empty()) memcpy(B.data() + H.off_x, ext.data(), 4 * ext.size());
    if (ns) memcpy(B.data() + H.off_meta, meta.data(), sizeof(int2) * ns);
    if (ns) memcpy(B.data() + H.off_srow, srow.data(), sizeof(short) * 32 * (size_t)ns);
    if (!hmeta.empty()) memcpy(B.data() + H.off_hmeta, hmeta.data(), 4 * hmeta.size());
    // local ids are encoded below, once the halo padding (and so the zero slot) is known;
    // keep what the encoder needs
    (void)order;
  }
  const int Lp = (lx_max + 3) & ~3;
  const int zero_id = R + Lp;
  const size_t floats = (size_t)6 * R + Lp + 4;
  const size_t smem = 4 * floats + blk_max;
  if (zero_id > 65535 || smem > smem_limit || R > 32767) return GN_OK;  // does not fit

  // encode the 16-bit local ids: own row r -> r, external halo t -> R + t, padding -> zero
  for (int b = 0; b < nb; ++b) {
    const int rb = part[b], re = part[b + 1];
    std::vector<unsigned char>& B = blocks[b];
    HaloHeader* H = reinterpret_cast<HaloHeader*>(B.data());
    H->zero_id = zero_id;
    const int* ext = reinterpret_cast<const int*>(B.data() + H->off_x);
    for (int t = 0; t < H->lx; ++t) {
      extpos[ext[t]] = t;
    }
    auto lid = [&](int j) -> uint16_t {
      return (uint16_t)((j >= rb && j < re) ? (j - rb) : (R + extpos[j]));
    };
    const int2* meta = reinterpret_cast<const int2*>(B.data() + H->off_meta);
    const short* srow = reinterpret_cast<const short*>(B.data() + H->off_srow);
    uint16_t* sell = reinterpret_cast<uint16_t*>(B.data() + H->off_sell);
    // Within a slice every lane's row may list its entries in any order.  Column by column,
    // give each lane the unused entry whose shared-memory bank (local id mod 32) is least
    // taken in that column, so the 32 lanes' gathers spread over the banks.
    std::vector<std::vector<uint16_t>> pending(32);
    for (int s = 0; s < H->ns; ++s) {
      for (int l = 0; l < 32; ++l) {
        const int r = srow[s * 32 + l];
        pending[l].clear();
        if (r >= 0)
          for (int64_t e = rp[rb + r]; e < rp[rb + r + 1]; ++e) pending[l].push_back(lid(ci[e]));
      }
      for (int k = 0; k < meta[s].y; ++k) {
        int load[32] = {0};
        for (int l = 0; l < 32; ++l) {
          std::vector<uint16_t>& q = pending[l];
          uint16_t pick = (uint16_t)zero_id;
          if (!q.empty()) {
            size_t best = 0;
            for (size_t t = 1; t < q.size() && load[q[best] & 31]; ++t)
              if (load[q[t] & 31] < load[q[best] & 31]) best = t;
            pick = q[best];
            q[best] = q.back();
            q.pop_back();
            ++load[pick & 31];
          }
          sell[meta[s].x + (k >> 2) * 128 + l * 4 + (k & 3)] = pick;
        }
      }
    }
    const int* hm = reinterpret_cast<const int*>(B.data() + H->off_hmeta);
    uint16_t* hl = reinterpret_cast<uint16_t*>(B.data() + H->off_hl);
    for (int h = 0; h < H->nheavy; ++h) {
      const int r = hm[3 * h], o = hm[3 * h + 1], d = hm[3 * h + 2];
      for (int k = 0; k < d; ++k) hl[o + k] = lid(ci[rp[rb + r] + k]);
    }
  }
  std::vector<int64_t> hoff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) hoff[b + 1] = hoff[b] + (int64_t)blocks[b].size();
  std::vector<unsigned char> blob((size_t)std::max<int64_t>(hoff[nb], 16));
  for (int b = 0; b < nb; ++b) memcpy(blob.data() + hoff[b], blocks[b].data(), blocks[b].size());
  GN_CUDA(cudaMalloc(&g->d_hoff, sizeof(int64_t) * (nb + 1)));
  GN_CUDA(cudaMalloc(&g->d_hblob, blob.size()));
  GN_CUDA(cudaMemcpyAsync(g->d_hoff, hoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaMemcpyAsync(g->d_hblob, blob.data(), blob.size(), cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  g->halo_pad = Lp;
  g->rows_pad_halo = R;
  g->smem_bytes = smem;
  *fits = true;
  return GN_OK;
}

const void* halo_kernel(int rows_pad) {
  return rows_pad <= 2 * kThreads ? (const void*)k_gn_halo<true> : (const void*)k_gn_halo<false>;
}

}  // namespace gn
