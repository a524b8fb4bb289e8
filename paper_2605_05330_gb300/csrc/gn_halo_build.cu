// gn_halo_build.cu -- host side of the halo gather mode: each CTA's halo list, the exchange
// (pull or push) and the packed per-CTA blocks (gn_halo.cuh) with their SELL-32 slices, heavy
// row chunks and send lists, uploaded once per graph.  The layout itself is described in
// gn_halo.cu.
#include <algorithm>
#include <climits>
#include <cstring>
#include <memory>
#include <numeric>
#include <vector>

#include "gn_halo.cuh"
#include "gn_internal.cuh"

namespace gn {

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
  int* elane = (cs.elane.resize(E), cs.elane.data());
  int* ebank = (cs.ebank.resize(E), cs.ebank.data());
  int* ecol = (cs.ecol.resize(E), cs.ecol.data());
  // the used-colour sets: on the stack for up to 64 colours (every slice in practice)
  uint64_t ul_small[32], ub_small[32];
  uint64_t* ul = ul_small;
  uint64_t* ub = ub_small;
  if (nw > 1) {
    cs.used_l.assign(32 * (size_t)nw, 0);
    cs.used_b.assign(32 * (size_t)nw, 0);
    ul = cs.used_l.data();
    ub = cs.used_b.data();
  } else {
    for (int i = 0; i < 32; ++i) ul_small[i] = ub_small[i] = 0;
  }
  const uint64_t last_mask = (W & 63) ? (1ull << (W & 63)) - 1 : ~0ull;  // colours < W in the last word
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
        const uint64_t both = ~(ul[(size_t)l * nw + w] | ub[(size_t)b * nw + w]) & (w + 1 < nw ? ~0ull : last_mask);
        if (both) a = w * 64 + __builtin_ctzll(both);
      }
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

// color_slice for up to 64 colours, on fixed-size arrays: the same edges in the same order, the
// same choices, so the same columns.  lid[l][0 .. nl[l]) lists lane l's ids; col[l][k] receives
// the column of lid[l][k]; ul[l] and ub[b] receive the colours used at lane l and at bank b.
struct ColorScratch64 {
  int16_t at_l[32 * 64], at_b[32 * 64];  // [vertex * W + colour] -> edge, or -1 (built on demand)
  uint8_t elane[32 * 64], ebank[32 * 64], ecol[32 * 64];
  int16_t path[32 * 64];
};
static void color_slice64(int W, const uint16_t (*lid)[64], const int* nl, uint8_t (*col)[64], ColorScratch64& cs,
                          uint64_t* ul, uint64_t* ub) {
  const uint64_t mask = W == 64 ? ~0ull : (1ull << W) - 1;
  for (int i = 0; i < 32; ++i) ul[i] = ub[i] = 0;
  bool tables = false;
  auto put = [&](int f, int x) {
    cs.ecol[f] = (uint8_t)x;
    ul[cs.elane[f]] |= 1ull << x;
    ub[cs.ebank[f]] |= 1ull << x;
    if (tables) {
      cs.at_l[cs.elane[f] * W + x] = (int16_t)f;
      cs.at_b[cs.ebank[f] * W + x] = (int16_t)f;
    }
  };
  // Lane l's colour set stays in a register while its entries are coloured: an alternating
  // path reaches lanes only through edges of colour a, which is free at l, so it never changes
  // lane l's set.
  int e = 0;
  for (int l = 0; l < 32; ++l) {
    uint64_t lu = 0;
    for (int k = 0; k < nl[l]; ++k, ++e) {
      const int b = lid[l][k] & 31;
      cs.elane[e] = (uint8_t)l;
      cs.ebank[e] = (uint8_t)b;
      const uint64_t both = ~(lu | ub[b]) & mask;
      if (both && !tables) {  // the lowest colour free at both ends
        const uint64_t bit = both & (0 - both);
        lu |= bit;
        ub[b] |= bit;
        cs.ecol[e] = (uint8_t)__builtin_ctzll(bit);
        continue;
      }
      ul[l] = lu;
      int a;
      if (both) {
        a = __builtin_ctzll(both);
      } else {
        if (!tables) {
          for (int i = 0; i < 32 * W; ++i) cs.at_l[i] = cs.at_b[i] = -1;
          for (int f = 0; f < e; ++f) {
            cs.at_l[cs.elane[f] * W + cs.ecol[f]] = (int16_t)f;
            cs.at_b[cs.ebank[f] * W + cs.ecol[f]] = (int16_t)f;
          }
          tables = true;
        }
        a = __builtin_ctzll(~ul[l]);
        const int c = __builtin_ctzll(~ub[b]);
        int np = 0, v = b, cur = a;
        bool bank_side = true;
        for (;;) {
          const int f = bank_side ? cs.at_b[v * W + cur] : cs.at_l[v * W + cur];
          if (f < 0) break;
          cs.path[np++] = (int16_t)f;
          v = bank_side ? cs.elane[f] : cs.ebank[f];
          bank_side = !bank_side;
          cur = cur == a ? c : a;
        }
        for (int q = 0; q < np; ++q) {  // the path's edges give up their colours
          const int f = cs.path[q], x = cs.ecol[f];
          cs.at_l[cs.elane[f] * W + x] = -1;
          cs.at_b[cs.ebank[f] * W + x] = -1;
          ul[cs.elane[f]] &= ~(1ull << x);
          ub[cs.ebank[f]] &= ~(1ull << x);
        }
        for (int q = 0; q < np; ++q) {
          const int f = cs.path[q];
          put(f, cs.ecol[f] == a ? c : a);
        }
      }
      put(e, a);
      lu = ul[l];
    }
    ul[l] = lu;
  }
  e = 0;
  for (int l = 0; l < 32; ++l)
    for (int k = 0; k < nl[l]; ++k) col[l][k] = cs.ecol[e++];
}

// A CTA's halo is "dense" when it averages at least this many values per 32-byte sector:
// then the pull exchange reads few sectors and wins; below it the push exchange does.
static constexpr double kPullDensity = 4.0;

// The halo mode's host side, in three steps:
//  - halo_lists: each CTA's distinct external neighbours (its halo), in increasing id order,
//    with the 32-byte sectors of the state vector they touch (the exchange is chosen by their
//    density);
//  - encode_halo_blocks: the packed per-CTA blocks for one exchange, in host memory;
//  - build_halo: both, for the exchange `want` (GN_GATHER_HALO: by the halo density;
//    GN_GATHER_HALO_PULL / _PUSH: that one), and the upload.  *fits = false (and nothing is
//    built on the device) when a CTA's working set does not fit shared memory or 16-bit local
//    ids; with the automatic choice the other exchange is tried before giving up.
// The per-CTA work runs on the host threads, a CTA at a time (parallel_items); every CTA's
// output is its own.
struct HaloBlocks {
  bool fits = false;
  int R = 0;                  // rows per CTA, padded to 4 (local ids of the halo start here)
  int Lp = 0;                 // the longest halo, padded to 4 (32 zero slots follow it)
  size_t smem = 0;            // dynamic shared memory of the kernel
  int64_t inbox_slots = 0;    // push: all CTAs' inbox slots
  std::vector<int64_t> hoff;  // [nblocks + 1] byte offsets of the blocks in blob
  std::unique_ptr<unsigned char[]> blob;
  size_t blob_bytes = 0;
};
static void halo_lists(int n, const std::vector<int32_t>& rp, const int32_t* ci, const std::vector<int32_t>& part,
                       std::vector<std::vector<int32_t>>& ext, int64_t* vals, int64_t* sectors);
static void encode_halo_blocks(int n, const std::vector<int32_t>& rp, const int32_t* ci,
                               const std::vector<int32_t>& part, const std::vector<std::vector<int32_t>>& ext,
                               bool push, size_t smem_limit, HaloBlocks* out);

// The slots of one send piece: m <= kSendPiece values (owner-local ids, bank = id & 31) in
// L = round4(m) slots.  The owner's warp stores slots 4j .. 4j + 3 from lane j (one 16-byte
// store) and gathers their values with four instructions, the u-th reading slot 4j + u of
// every lane, so the placement decides the bank conflicts of the gathers.  The rule is a
// greedy over the values of the busiest banks first (ties by bank, then by value index): each
// goes to the instruction u that has a free lane and does not yet read its bank, the least
// loaded such u first, ties to the lowest u (any u with a free lane, least loaded first, when
// every one reads it).  place[s] = the index of the value in slot s, or -(1 + bank) for
// padding, bank being one that no value of that instruction reads (where there is one).
// Returns L.
//
// That greedy is a round robin.  A bank's values are placed together, so at a bank's start no
// instruction reads it yet.  The counts (ordered by count, then u) then always read "the
// first p instructions hold c + 1 values, the others c", and the least loaded are p, p + 1, ...
// mod 4.  So the j-th value in bank order goes to instruction j mod 4, whose count is then
// j / 4 < L / 4: no instruction is full when its turn comes.
static int place_piece(const int32_t* lid, int m, int* place) {
  const int L = (m + 3) & ~3, lanes = L / 4;
  // the banks by decreasing load, ties by bank (a counting sort on maxl - load)
  int load[32] = {0}, maxl = 0;
  for (int i = 0; i < m; ++i) ++load[lid[i] & 31];
  for (int b = 0; b < 32; ++b) maxl = std::max(maxl, load[b]);
  int nat[kSendPiece + 2], border[32];
  for (int v = 0; v <= maxl + 1; ++v) nat[v] = 0;
  for (int b = 0; b < 32; ++b) ++nat[maxl - load[b] + 1];
  for (int v = 1; v <= maxl + 1; ++v) nat[v] += nat[v - 1];
  for (int b = 0; b < 32; ++b) border[nat[maxl - load[b]]++] = b;
  // each bank's first rank in that order, and the instructions its ranks a .. a + load - 1 go
  // to (all four from a load of 4 up): the banks each instruction reads
  int rank[32];
  uint32_t used[4] = {0, 0, 0, 0};
  for (int r = 0, a = 0; r < 32; ++r) {
    const int b = border[r], l = load[b];
    rank[b] = a;
    const unsigned x = ((1u << std::min(l, 4)) - 1) << (a & 3), w = (x | x >> 4) & 15u;
    for (int u = 0; u < 4; ++u) used[u] |= ((w >> u) & 1u) << b;
    a += l;
  }
  // the values in index order: each to instruction (its rank) mod 4, at that instruction's next
  // lane (four 16-bit lane counters in one word)
  uint64_t pos = 0;
  for (int i = 0; i < m; ++i) {
    const int u = rank[lid[i] & 31]++ & 3, sh = 16 * u;
    place[4 * (int)((pos >> sh) & 0xffff) + u] = i;
    pos += 1ull << sh;
  }
  // instructions m mod 4 .. 3 hold one value fewer: their last lane is padding
  for (int u = m & 3; u != 0 && u < 4; ++u) {
    const int zb = used[u] == 0xffffffffu ? 0 : __builtin_ctz(~used[u]);
    place[4 * (lanes - 1) + u] = -1 - zb;
  }
  return L;
}

gn_status build_halo(gn_graph* g, const std::vector<int32_t>& rp, const int32_t* ci,
                     const std::vector<int32_t>& part, size_t smem_limit, int want, bool* fits) {
  *fits = false;
  const int nb = (int)part.size() - 1;
  const int n = g->n;
  std::vector<std::vector<int32_t>> ext(nb);
  int64_t vals = 0, sectors = 0;
  halo_lists(n, rp, ci, part, ext, &vals, &sectors);
  // the exchange: forced, or by the density of the halos in memory
  bool push = want == GN_GATHER_HALO_PUSH ||
              (want == GN_GATHER_HALO && (double)vals < kPullDensity * (double)std::max<int64_t>(sectors, 1));
  HaloBlocks hb;
  encode_halo_blocks(n, rp, ci, part, ext, push, smem_limit, &hb);
  if (!hb.fits && want == GN_GATHER_HALO) {  // the automatic choice tries the other exchange
    push = !push;
    encode_halo_blocks(n, rp, ci, part, ext, push, smem_limit, &hb);
  }
  if (!hb.fits) return GN_OK;
  GN_CUDA(cudaMalloc(&g->d_hoff, sizeof(int64_t) * (nb + 1)));
  GN_CUDA(cudaMalloc(&g->d_hblob, hb.blob_bytes));
  // the exchange buffers: push, the inboxes; pull, one slot per vertex (read by the tagged
  // exchange only); three of each (two alternate under the barrier or the flags, three rotate
  // in the tagged exchange)
  g->inbox_len = push ? std::max<int64_t>(hb.inbox_slots, 4) : (int64_t)((n + 3) & ~3);
  GN_CUDA(cudaMalloc(&g->d_inbox, sizeof(float) * 3 * (size_t)g->inbox_len));
  GN_CUDA(cudaMemsetAsync(g->d_inbox, 0, sizeof(float) * 3 * (size_t)g->inbox_len, g->stream));
  g->halo_push = push;
  GN_CUDA(cudaMemcpyAsync(g->d_hoff, hb.hoff.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice,
                          g->stream));
  GN_CUDA(cudaMemcpyAsync(g->d_hblob, hb.blob.get(), hb.blob_bytes, cudaMemcpyHostToDevice, g->stream));
  GN_CUDA(cudaStreamSynchronize(g->stream));
  g->halo_pad = hb.Lp;
  g->rows_pad_halo = hb.R;
  g->smem_bytes = hb.smem;
  *fits = true;
  return GN_OK;
}

// The halo lists, from a bitmap of the vertex range per host thread (a mark per entry, then a
// scan of the marked words).
static void halo_lists(int n, const std::vector<int32_t>& rp, const int32_t* ci, const std::vector<int32_t>& part,
                       std::vector<std::vector<int32_t>>& ext, int64_t* vals, int64_t* sectors) {
  const int nb = (int)part.size() - 1;
  std::vector<int64_t> sectors_of(nb, 0);
  std::vector<std::vector<uint64_t>> bitmaps(host_threads());  // per host thread, kept all-zero
  parallel_items(nb, [&](int b, int t) {
    std::vector<uint64_t>& bits = bitmaps[t];
    if (bits.empty()) bits.assign((size_t)n / 64 + 1, 0);
    {
      const int rb = part[b], re = part[b + 1];
      // every entry marked (no branch per entry), then the CTA's own rows unmarked
      int wlo = INT32_MAX, whi = -1;
      for (int64_t e = rp[rb]; e < rp[re]; ++e) {
        const int j = ci[e];
        bits[j >> 6] |= 1ull << (j & 63);
        wlo = std::min(wlo, j >> 6);
        whi = std::max(whi, j >> 6);
      }
      if (re > rb) {
        const int w0 = rb >> 6, w1 = (re - 1) >> 6;
        const uint64_t lo = ~0ull << (rb & 63), hi = ~0ull >> (63 - ((re - 1) & 63));
        if (w0 == w1) {
          bits[w0] &= ~(lo & hi);
        } else {
          bits[w0] &= ~lo;
          for (int wd = w0 + 1; wd < w1; ++wd) bits[wd] = 0;
          bits[w1] &= ~hi;
        }
      }
      std::vector<int32_t>& xb = ext[b];
      size_t count = 0;
      for (int wd = wlo; wd <= whi; ++wd) count += (size_t)__builtin_popcountll(bits[wd]);
      xb.resize(count);
      int32_t* out = xb.data();
      // a sector is 8 vertices, one byte of the bitmap: the sectors touched are its nonzero bytes
      constexpr uint64_t k7f = 0x7f7f7f7f7f7f7f7full;
      int64_t sec = 0;
      for (int wd = wlo; wd <= whi; ++wd) {
        uint64_t m = bits[wd];
        bits[wd] = 0;
        sec += __builtin_popcountll((((m & k7f) + k7f) | m) & ~k7f);
        while (m) {
          *out++ = wd * 64 + __builtin_ctzll(m);
          m &= m - 1;
        }
      }
      sectors_of[b] = sec;
    }
  });
  *vals = 0;
  *sectors = 0;
  for (int b = 0; b < nb; ++b) {
    *vals += (int64_t)ext[b].size();
    *sectors += sectors_of[b];
  }
}

// The blocks for one exchange (see build_halo).
static void encode_halo_blocks(int n, const std::vector<int32_t>& rp, const int32_t* ci,
                               const std::vector<int32_t>& part, const std::vector<std::vector<int32_t>>& ext,
                               bool push, size_t smem_limit, HaloBlocks* out) {
  out->fits = false;
  const int nb = (int)part.size() - 1;
  int max_rows = 0;
  for (int b = 0; b < nb; ++b) max_rows = std::max(max_rows, part[b + 1] - part[b]);
  const int R = (max_rows + 3) & ~3;

  // Push: each consumer's inbox.  Consumer c's halo (ext[c], sorted by id) holds the values of
  // one owner CTA as one run (the partition is contiguous); in the inbox each run starts at a
  // multiple of 4 slots and is padded to one, and its pieces of kSendPiece slots are placed by
  // place_piece.  The owner o sends its runs consumer by consumer: a piece (first inbox slot,
  // length, first source, 0) per kSendPiece slots from each run's start, and the source id of
  // every slot (the owner-local id read, or for padding the zero slot of the bank place_piece
  // names).  hslot: the inbox slot (within c's region) of ext[c][t].  Pull: the halo in ext
  // order, 4-slot aligned regions.
  struct Sends {
    std::vector<int4> pieces;  // all four fields multiples of 4 (but the last)
    std::vector<uint16_t> src;
  };
  std::vector<Sends> sends(nb);
  std::vector<std::vector<int32_t>> hslot(nb);
  std::vector<int64_t> lxp(nb), inbox_off(nb + 1, 0);
  std::vector<std::vector<int2>> hrun(push ? nb : 0);  // push: each consumer's runs
  if (push) {
    // each consumer's runs, (owner, padded length) in owner order
    parallel_items(nb, [&](int c, int) {
      const std::vector<int32_t>& xc = ext[c];
      std::vector<int2>& runs = hrun[c];
      runs.clear();
      int64_t total = 0;
      for (size_t t = 0, o = 0; t < xc.size();) {
        while (xc[t] >= part[o + 1]) ++o;
        size_t e = t;
        while (e < xc.size() && xc[e] < part[o + 1]) ++e;
        const int len = (int)((e - t + 3) & ~(size_t)3);
        runs.push_back(make_int2((int)o, len));
        total += len;
        t = e;
      }
      lxp[c] = total;
    });
  } else {
    for (int c = 0; c < nb; ++c) lxp[c] = (int64_t)ext[c].size();
  }
  // local ids: own rows below R, halo slots from R, then 32 zero slots (one per bank) after the
  // longest halo padded to 4
  int64_t lx_max = 0;
  for (int c = 0; c < nb; ++c) lx_max = std::max(lx_max, lxp[c]);
  if (lx_max > 65535) return;  // does not fit 16-bit local ids
  const int Lp = (int)((lx_max + 3) & ~(int64_t)3);
  const int zero_id = R + Lp;
  if (push) {
    for (int c = 0; c < nb; ++c) inbox_off[c + 1] = inbox_off[c] + lxp[c];
    if (inbox_off[nb] > (int64_t)INT32_MAX) return;  // inbox slots do not fit 32 bits
    // where each run goes in its owner's lists: consumers in order
    std::vector<std::vector<int2>> roff(nb);  // per consumer and run: (first source, first piece)
    std::vector<int64_t> scount(nb, 0), pcount(nb, 0);
    for (int c = 0; c < nb; ++c) {
      roff[c].resize(hrun[c].size());
      for (size_t j = 0; j < hrun[c].size(); ++j) {
        const int o = hrun[c][j].x, len = hrun[c][j].y;
        roff[c][j] = make_int2((int)scount[o], (int)pcount[o]);
        scount[o] += len;
        pcount[o] += (len + kSendPiece - 1) / kSendPiece;
      }
    }
    parallel_items(nb, [&](int o, int) {
      sends[o].src.resize(scount[o]);
      sends[o].pieces.resize(pcount[o]);
    });
    // the placement, written straight into the owners' lists (disjoint ranges per consumer)
    parallel_items(nb, [&](int c, int) {
      const std::vector<int32_t>& xc = ext[c];
      std::vector<int32_t>& hs = hslot[c];
      hs.resize(xc.size());
      int32_t lid[kSendPiece];
      int place[kSendPiece];
      int slot = 0;
      size_t j = 0;
      for (size_t t = 0, o = 0; t < xc.size(); ++j) {
        while (xc[t] >= part[o + 1]) ++o;
        size_t e = t;
        while (e < xc.size() && xc[e] < part[o + 1]) ++e;
        Sends& so = sends[o];
        int soff = roff[c][j].x, poff = roff[c][j].y;
        for (size_t a = t; a < e; a += kSendPiece) {
          const int m = (int)std::min<size_t>(kSendPiece, e - a);
          for (int i = 0; i < m; ++i) lid[i] = xc[a + i] - part[o];
          const int L = place_piece(lid, m, place);
          so.pieces[poff++] = make_int4((int)(inbox_off[c] + slot), L, soff, 0);
          uint16_t* sp = so.src.data() + soff;
          for (int q = 0; q < L; ++q) {
            const int i = place[q];
            if (i >= 0) {
              sp[q] = (uint16_t)lid[i];
              hs[a + i] = slot + q;
            } else {
              sp[q] = (uint16_t)(zero_id + (((-1 - i) - zero_id) & 31));
            }
          }
          slot += L;
          soff += L;
        }
        t = e;
      }
    });
  } else {
    for (int c = 0; c < nb; ++c) inbox_off[c + 1] = inbox_off[c] + ((lxp[c] + 3) & ~(int64_t)3);
  }

  // pass 1, per CTA: rows into interior / boundary / heavy, slices, chunks, send pieces and
  // the block layout (the plan; pass 2 writes the blocks straight into the upload buffer)
  struct Plan {
    HaloHeader H;
    std::vector<int2> meta;
    std::vector<short> srow;
    std::vector<int> hmeta, hchunk;
    std::vector<int32_t> dep;
    std::vector<int4> pieces;
    std::vector<uint16_t> src;
  };
  std::vector<Plan> plans(nb);
  parallel_items(nb, [&](int b, int) {
    {
      const int rb = part[b], re = part[b + 1], nr = re - rb;
      const std::vector<int32_t>& xb = ext[b];
      // the CTAs owning the halo (xb is sorted and the partition contiguous: one walk)
      std::vector<int32_t> dep;
      for (size_t t = 0, o = 0; t < xb.size(); ++t) {
        while (xb[t] >= part[o + 1]) ++o;
        if (dep.empty() || dep.back() != (int32_t)o) dep.push_back((int32_t)o);
      }
      std::vector<int> light_int, light_bnd, heavy;
      for (int r = 0; r < nr; ++r) {
        const int64_t a = rp[rb + r], c = rp[rb + r + 1];
        if (c - a > kHeavyHalo) {
          heavy.push_back(r);
          continue;
        }
        // a row's entries are increasing, so it reads another CTA's row iff its first or last does
        const bool bnd = c > a && (ci[a] < rb || ci[c - 1] >= re);
        (bnd ? light_bnd : light_int).push_back(r);
      }
      // by degree, descending, then by row (the lists are in row order and light degrees are at
      // most kHeavyHalo, so a stable counting sort)
      auto by_deg = [&](std::vector<int>& v) {
        int at[kHeavyHalo + 2] = {0};
        for (int r : v) ++at[kHeavyHalo - (int)(rp[rb + r + 1] - rp[rb + r]) + 1];
        for (int d = 1; d <= kHeavyHalo + 1; ++d) at[d] += at[d - 1];
        std::vector<int> out(v.size());
        for (int r : v) out[at[kHeavyHalo - (int)(rp[rb + r + 1] - rp[rb + r])]++] = r;
        v.swap(out);
      };
      by_deg(light_int);
      by_deg(light_bnd);
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
      H.lx = (int)lxp[b];
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
      std::vector<int4> pieces = std::move(sends[b].pieces);
      std::vector<uint16_t> src = std::move(sends[b].src);
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
      Plan& P = plans[b];
      P.H = H;
      P.meta = std::move(meta);
      P.srow = std::move(srow);
      P.hmeta = std::move(hmeta);
      P.hchunk = std::move(hchunk);
      P.dep = std::move(dep);
      P.pieces = std::move(pieces);
      P.src = std::move(src);
    }
  });
  size_t blk_max = 0;
  for (int b = 0; b < nb; ++b) blk_max = std::max(blk_max, (size_t)plans[b].H.bytes);
  const size_t floats = (size_t)6 * R + Lp + 32;
  const size_t smem = 4 * floats + blk_max;
  if (zero_id + 31 > 65535 || smem > smem_limit || R > 32767) return;  // does not fit
  std::vector<int64_t> hoff(nb + 1, 0);
  for (int b = 0; b < nb; ++b) hoff[b + 1] = hoff[b] + plans[b].H.bytes;
  const size_t blob_bytes = (size_t)std::max<int64_t>(hoff[nb], 16);
  std::unique_ptr<unsigned char[]> blob(new unsigned char[blob_bytes]);

  // pass 2, per CTA: the 16-bit local ids (own row r -> r, external vertex -> R + its halo
  // slot, padding -> a zero slot)
  struct EncodeScratch {
    std::unique_ptr<uint16_t[]> lidtab;  // local id of each vertex the CTA reads (set before it is read)
    std::vector<uint16_t> lids[32];
    std::vector<int> cols[32];
    ColorScratch cs;
    std::vector<uint16_t> bucket[32];
    // a slice on fixed-size arrays (every light row has at most kHeavyHalo = 64 entries)
    uint16_t lidA[32][64];
    int nl[32];
    uint8_t colA[32][64];
    uint8_t extra[32 * 64];  // per (bank, column): folded entries placed there (zero between slices)
    uint16_t fold[32 * 64];
    ColorScratch64 cs64;
  };
  std::vector<EncodeScratch> scratch(host_threads());
  for (EncodeScratch& X : scratch) memset(X.extra, 0, sizeof X.extra);
  parallel_items(nb, [&](int b, int t) {
    EncodeScratch& X = scratch[t];
    if (!X.lidtab) X.lidtab.reset(new uint16_t[std::max(n, 1)]);
    uint16_t* lidtab = X.lidtab.get();
    std::vector<uint16_t>* lids = X.lids;
    std::vector<int>* cols = X.cols;
    ColorScratch& cs = X.cs;
    uint8_t* extra = X.extra;
    uint16_t(*lidA)[64] = X.lidA;
    int* nl = X.nl;
    uint8_t(*colA)[64] = X.colA;
    uint16_t* fold = X.fold;
    uint64_t usedcols[32];
    std::vector<uint16_t>* bucket = X.bucket;
    {
      const int rb = part[b], re = part[b + 1];
      // the block: zeros, then the plan's header and sections
      unsigned char* B = blob.get() + hoff[b];
      {
        const Plan& P = plans[b];
        const HaloHeader& PH = P.H;
        memset(B, 0, PH.bytes);
        memcpy(B, &PH, sizeof PH);
        if (PH.ns) memcpy(B + PH.off_meta, P.meta.data(), sizeof(int2) * PH.ns);
        if (PH.ns) memcpy(B + PH.off_srow, P.srow.data(), sizeof(short) * 32 * (size_t)PH.ns);
        if (!P.hmeta.empty()) memcpy(B + PH.off_hmeta, P.hmeta.data(), 4 * P.hmeta.size());
        if (!P.dep.empty()) memcpy(B + PH.off_dep, P.dep.data(), 4 * P.dep.size());
        if (!P.hchunk.empty()) memcpy(B + PH.off_hchunk, P.hchunk.data(), 4 * P.hchunk.size());
        if (!P.pieces.empty()) memcpy(B + PH.off_piece, P.pieces.data(), sizeof(int4) * P.pieces.size());
        if (!P.src.empty()) memcpy(B + PH.off_src, P.src.data(), 2 * P.src.size());
        if (!push && !ext[b].empty()) memcpy(B + PH.off_x, ext[b].data(), 4 * ext[b].size());
      }
      HaloHeader* H = reinterpret_cast<HaloHeader*>(B);
      H->zero_id = zero_id;
      // a vertex's local id is one table read (own rows below R, halo slots from R; no branch
      // per entry; every id fits 16 bits, zero_id + 31 <= 65535 was checked)
      for (size_t t = 0; t < ext[b].size(); ++t)
        lidtab[ext[b][t]] = (uint16_t)(R + (push ? hslot[b][t] : (int32_t)t));
      for (int j = rb; j < re; ++j) lidtab[j] = (uint16_t)(j - rb);
      auto lid = [&](int j) -> uint16_t { return lidtab[j]; };
      const int2* meta = reinterpret_cast<const int2*>(B + H->off_meta);
      const short* srow = reinterpret_cast<const short*>(B + H->off_srow);
      uint16_t* sell = reinterpret_cast<uint16_t*>(B + H->off_sell);
      // Every lane's row may list its entries in any order: colour the slice (color_slice) so
      // that each column's real entries lie in distinct banks, then pad each lane's empty
      // columns with the zero slot of a bank no real entry of that column uses (all padding of
      // a column reads that one address: a broadcast).
      static_assert(kHeavyHalo <= 64, "a light row's entries fit one 64-bit column set");
      for (int s = 0; s < H->ns; ++s) {
        const int W = meta[s].y;
        int load[32] = {0};
        for (int l = 0; l < 32; ++l) {
          const int r = srow[s * 32 + l];
          int m = 0;
          if (r >= 0)
            for (int64_t e = rp[rb + r]; e < rp[rb + r + 1]; ++e) {
              const uint16_t id = lid(ci[e]);
              lidA[l][m++] = id;
              ++load[id & 31];
            }
          nl[l] = m;
        }
        // colours for the slice's busiest bank; when that is more than the slice's width, the
        // colours past the width fold into each lane's free columns, least-used bank first
        // (only those gathers can conflict)
        int Wc = W;
        for (int t = 0; t < 32; ++t) Wc = std::max(Wc, load[t]);
        uint64_t ul[32], ub[32];
        const uint64_t wmask = W == 64 ? ~0ull : (1ull << W) - 1;
        uint32_t foldlanes = 0;  // the lanes with a colour from W up
        if (Wc <= 64) {
          color_slice64(Wc, lidA, nl, colA, X.cs64, ul, ub);
          for (int l = 0; l < 32; ++l) foldlanes |= (ul[l] & ~wmask) ? 1u << l : 0u;
        } else {  // more than 64 colours: the general version
          for (int l = 0; l < 32; ++l) lids[l].assign(lidA[l], lidA[l] + nl[l]);
          color_slice(Wc, lids, cols, cs);
          for (int l = 0; l < 32; ++l) ul[l] = ub[l] = 0;
          for (int l = 0; l < 32; ++l)
            for (int k = 0; k < nl[l]; ++k) {
              colA[l][k] = (uint8_t)std::min(cols[l][k], 255);
              if (cols[l][k] >= W) foldlanes |= 1u << l;
              if (cols[l][k] < 64) {  // colours from 64 up are all folded below (W <= 64)
                ul[l] |= 1ull << cols[l][k];
                ub[lidA[l][k] & 31] |= 1ull << cols[l][k];
              }
            }
        }
        if (Wc > W) {
          // The colouring is proper, so below the width bank bk holds column c at most once: the
          // bit c of ub[bk].  A folded entry (colour from W up; lane order, then entry order)
          // takes the free column of its lane that its bank uses least, lowest first.  The
          // columns a bank uses no time (fresh) and exactly once (once) are bit sets, so the
          // lowest candidate comes from one of them; only columns used twice or more need the
          // counts (the bit plus the folded entries already placed there, in extra).
          uint64_t fresh[32], once[32], used[32];
          for (int t = 0; t < 32; ++t) {
            fresh[t] = ~ub[t] & wmask;
            once[t] = ub[t] & wmask;
            used[t] = ul[t] & wmask;
          }
          int nfold = 0;
          for (int l = 0; l < 32; ++l) {
            if (!(foldlanes >> l & 1u)) continue;  // nothing of lane l to fold
            for (int k = 0; k < nl[l]; ++k)
              if (colA[l][k] >= W) fold[nfold++] = (uint16_t)(l * 64 + k);
          }
          for (int q = 0; q < nfold; ++q) {
            const int l = fold[q] >> 6, k = fold[q] & 63, bk = lidA[l][k] & 31;
            const uint64_t freecols = ~used[l] & wmask;
            int best;
            if (freecols & fresh[bk]) {
              best = __builtin_ctzll(freecols & fresh[bk]);
            } else if (freecols & once[bk]) {
              best = __builtin_ctzll(freecols & once[bk]);
            } else {
              best = -1;
              int bo = INT_MAX;
              for (int c = 0; c < W; ++c) {
                if (!(freecols >> c & 1ull)) continue;
                const int o = (int)(ub[bk] >> c & 1ull) + extra[bk * 64 + c];
                if (o < bo) {
                  bo = o;
                  best = c;
                }
              }
            }
            const uint64_t bit = 1ull << best;
            colA[l][k] = (uint8_t)best;
            used[l] |= bit;
            if (fresh[bk] & bit) {  // 0 -> 1
              fresh[bk] &= ~bit;
              once[bk] |= bit;
            } else {  // 1 -> 2, or more
              once[bk] &= ~bit;
            }
            ++extra[bk * 64 + best];
          }
          for (int q = 0; q < nfold; ++q) extra[(lidA[fold[q] >> 6][fold[q] & 63] & 31) * 64 + colA[fold[q] >> 6][fold[q] & 63]] = 0;
        }
        // the real entries, each lane's used columns and each column's used banks; then the
        // padding: an empty slot of column k reads the zero slot of the lowest bank no real entry
        // of k uses (a column without a free bank has all 32 lanes real, so no empty slot)
        uint32_t colbanks[64] = {0};
        const int base = meta[s].x;
        for (int l = 0; l < 32; ++l) {
          uint64_t used = 0;
          for (int t = 0; t < nl[l]; ++t) {
            const int k = colA[l][t];
            sell[base + (k >> 2) * 128 + l * 4 + (k & 3)] = lidA[l][t];
            used |= 1ull << k;
            colbanks[k] |= 1u << (lidA[l][t] & 31);
          }
          usedcols[l] = used;
        }
        for (int l = 0; l < 32; ++l) {
          uint64_t empty = ~usedcols[l] & (W == 64 ? ~0ull : (1ull << W) - 1);
          while (empty) {
            const int k = __builtin_ctzll(empty);
            empty &= empty - 1;
            const int zb = __builtin_ctz(~colbanks[k]);
            sell[base + (k >> 2) * 128 + l * 4 + (k & 3)] = (uint16_t)(zero_id + ((zb - zero_id) & 31));
          }
        }
      }
      const int* hm = reinterpret_cast<const int*>(B + H->off_hmeta);
      const int* hc = reinterpret_cast<const int*>(B + H->off_hchunk);
      uint16_t* hl = reinterpret_cast<uint16_t*>(B + H->off_hl);
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
  out->R = R;
  out->Lp = Lp;
  out->smem = smem;
  out->inbox_slots = push ? inbox_off[nb] : 0;
  out->hoff = std::move(hoff);
  out->blob = std::move(blob);
  out->blob_bytes = blob_bytes;
  out->fits = true;
}

}  // namespace gn
