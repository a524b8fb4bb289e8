// Host-side checks of the halo block builder (gn_halo_build.cu, included here for its
// file-local functions), linked against libgn.so for the rest: the slice colouring, the
// send-piece placement (slot for slot against its rule written out plainly), the halo lists,
// and the decoded blocks of both exchanges on random graphs.  No GPU is used.  Prints "ok" and returns 0 when every check passes; prints what
// failed and returns 1 otherwise.
#include <algorithm>
#include <cstdio>
#include <random>
#include <vector>

#include "gn_halo_build.cu"

static int failures = 0;
#define CHECK(cond, what)                \
  do {                                   \
    if (!(cond)) {                       \
      if (failures < 20) std::printf("FAILED: %s\n", what); \
      ++failures;                        \
    }                                    \
  } while (0)

// A random slice: 32 lanes of at most W entries each (W <= 64), ids drawn from [0, span); skewed
// draws put many entries on a few banks.
static void random_slice(std::mt19937& rng, int W, int span, bool skew, uint16_t (*lid)[64], int* nl) {
  for (int l = 0; l < 32; ++l) {
    nl[l] = (int)(rng() % (unsigned)(W + 1));
    for (int k = 0; k < nl[l]; ++k) {
      unsigned id = rng() % (unsigned)span;
      if (skew && rng() % 4 == 0) id = (id & ~31u) | (rng() % 3);  // banks 0..2 get extra load
      lid[l][k] = (uint16_t)id;
    }
  }
}

static void check_colouring(std::mt19937& rng) {
  gn::ColorScratch cs;
  static gn::ColorScratch64 cs64;
  uint16_t lid[32][64];
  int nl[32];
  uint8_t col[32][64];
  std::vector<uint16_t> lv[32];
  std::vector<int> cv[32];
  for (int t = 0; t < 20000; ++t) {
    const int W = 4 * (1 + (int)(rng() % 16));  // slice widths 4 .. 64
    random_slice(rng, W, 32 + (int)(rng() % 8000), t % 3 == 0, lid, nl);
    int load[32] = {0};
    for (int l = 0; l < 32; ++l)
      for (int k = 0; k < nl[l]; ++k) ++load[lid[l][k] & 31];
    int Wc = W;
    for (int b = 0; b < 32; ++b) Wc = std::max(Wc, load[b]);
    if (Wc > 64) continue;  // the general version's own case
    uint64_t ul[32], ub[32];
    gn::color_slice64(Wc, lid, nl, col, cs64, ul, ub);
    for (int l = 0; l < 32; ++l) lv[l].assign(lid[l], lid[l] + nl[l]);
    gn::color_slice(Wc, lv, cv, cs);
    bool same = true, proper = true, sets = true;
    uint64_t lane_cols[32] = {0}, bank_cols[32] = {0};
    for (int l = 0; l < 32; ++l)
      for (int k = 0; k < nl[l]; ++k) {
        const int c = col[l][k], b = lid[l][k] & 31;
        same = same && c == cv[l][k];
        proper = proper && c < Wc && !(lane_cols[l] >> c & 1ull) && !(bank_cols[b] >> c & 1ull);
        lane_cols[l] |= 1ull << c;
        bank_cols[b] |= 1ull << c;
      }
    for (int i = 0; i < 32; ++i) sets = sets && ul[i] == lane_cols[i] && ub[i] == bank_cols[i];
    CHECK(same, "the 64-colour colouring gives the general colouring's columns");
    CHECK(proper, "the colouring is proper (distinct colours at each lane and each bank, below the width)");
    CHECK(sets, "the reported lane and bank colour sets are the colours used");
  }
}

// The send-piece rule written out as stated: values of the busiest banks first (ties by bank,
// then by index), each to the instruction with a free lane that does not yet read its bank, the
// least loaded such first, ties to the lowest; when every instruction with a free lane reads it,
// the least loaded of those.  Lanes of an instruction in value order; padding names the lowest
// bank the instruction does not read.
static int greedy_placement(const int32_t* lid, int m, int* place) {
  const int L = (m + 3) & ~3, lanes = L / 4;
  std::vector<int> order(m);
  for (int i = 0; i < m; ++i) order[i] = i;
  int load[32] = {0};
  for (int i = 0; i < m; ++i) ++load[lid[i] & 31];
  std::sort(order.begin(), order.end(), [&](int a, int b) {
    const int ba = lid[a] & 31, bb = lid[b] & 31;
    if (load[ba] != load[bb]) return load[ba] > load[bb];
    if (ba != bb) return ba < bb;
    return a < b;
  });
  std::vector<int> uof(m);
  int cnt[4] = {0, 0, 0, 0};
  uint32_t reads[4] = {0, 0, 0, 0};
  for (int i : order) {
    const int bk = lid[i] & 31;
    int best = -1;
    for (int pass = 0; pass < 2 && best < 0; ++pass)
      for (int u = 0; u < 4; ++u) {
        if (cnt[u] >= lanes || (pass == 0 && (reads[u] >> bk & 1u))) continue;
        if (best < 0 || cnt[u] < cnt[best]) best = u;
      }
    uof[i] = best;
    ++cnt[best];
    reads[best] |= 1u << bk;
  }
  int next[4] = {0, 0, 0, 0};
  for (int i = 0; i < m; ++i) place[4 * next[uof[i]]++ + uof[i]] = i;
  for (int u = 0; u < 4; ++u) {
    int zb = 0;
    while (zb < 32 && (reads[u] >> zb & 1u)) ++zb;
    if (zb == 32) zb = 0;
    for (int j = next[u]; j < lanes; ++j) place[4 * j + u] = -1 - zb;
  }
  return L;
}

static void check_placement(std::mt19937& rng) {
  int32_t lid[gn::kSendPiece];
  int place[gn::kSendPiece];
  for (int t = 0; t < 100000; ++t) {
    const int m = 1 + (int)(rng() % gn::kSendPiece);
    const int span = 32 + (int)(rng() % 5000);
    const unsigned crowd = t % 3 == 0 ? 1 + rng() % 4 : 0;  // a few banks take many of the values
    for (int i = 0; i < m; ++i) {
      lid[i] = (int32_t)(rng() % (unsigned)span);
      if (crowd && rng() % 2) lid[i] = (lid[i] & ~31) | (int32_t)(rng() % crowd);
    }
    const int L = gn::place_piece(lid, m, place);
    CHECK(L == ((m + 3) & ~3), "a piece takes m rounded up to 4 slots");
    int want[gn::kSendPiece];
    greedy_placement(lid, m, want);
    bool same = true;
    for (int q = 0; q < L; ++q) same = same && place[q] == want[q];
    CHECK(same, "the placement is the stated greedy's, slot for slot");
    std::vector<int> seen(m, 0);
    bool ok = true;
    uint32_t banks[4] = {0, 0, 0, 0};
    for (int q = 0; q < L; ++q)
      if (place[q] >= 0) {
        ok = ok && place[q] < m;
        if (place[q] < m) {
          ++seen[place[q]];
          banks[q & 3] |= 1u << (lid[place[q]] & 31);
        }
      }
    for (int i = 0; i < m; ++i) ok = ok && seen[i] == 1;
    CHECK(ok, "every value of a piece in exactly one slot");
    bool pad = true;
    for (int q = 0; q < L; ++q)
      if (place[q] < 0) {
        const int bank = -1 - place[q];
        pad = pad && bank >= 0 && bank < 32 && (banks[q & 3] == 0xffffffffu || !(banks[q & 3] >> bank & 1u));
      }
    CHECK(pad, "padding reads a bank that its gather's values leave free, where one is free");
  }
}

// A random simple graph: each vertex i draws neighbours within a window around i (locality, so
// interior rows and dense halos occur) or anywhere (cut edges), a few hubs draw hundreds
// (heavy rows); symmetrised, deduplicated and sorted.
static void random_graph(std::mt19937& rng, int n, int deg, int window, int hubs, std::vector<int32_t>& rp,
                         std::vector<int32_t>& ci) {
  std::vector<std::vector<int32_t>> adj(n);
  for (int i = 0; i < n; ++i) {
    const int d = i < hubs ? 150 + (int)(rng() % 300) : (int)(rng() % (2 * deg + 1));
    for (int t = 0; t < d; ++t) {
      int j = (window > 0 && rng() % 4 != 0) ? i - window + (int)(rng() % (2 * window + 1)) : (int)(rng() % n);
      if (j < 0 || j >= n || j == i) continue;
      adj[i].push_back(j);
      adj[j].push_back(i);
    }
  }
  rp.assign(n + 1, 0);
  ci.clear();
  for (int i = 0; i < n; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    adj[i].erase(std::unique(adj[i].begin(), adj[i].end()), adj[i].end());
    ci.insert(ci.end(), adj[i].begin(), adj[i].end());
    rp[i + 1] = (int32_t)ci.size();
  }
}

// Decodes every CTA's block and checks what the kernel relies on: each row is summed once (a
// SELL lane or a heavy row), its real ids name exactly its neighbours (own rows, halo slots whose
// value is the right vertex's, through the pull list or the owners' send lists), everything else
// reads a zero slot, padding in a SELL column reads a bank no real entry of that column reads,
// interior slices read no halo, the dependency list names the halo's owners, and in push mode
// the owners' send pieces fill every inbox slot once.
static void check_blocks(const char* name, int n, const std::vector<int32_t>& rp, const std::vector<int32_t>& ci,
                         int nb, bool push) {
  std::vector<int32_t> part(nb + 1);
  for (int b = 0; b <= nb; ++b) part[b] = (int32_t)((int64_t)n * b / nb);
  std::vector<std::vector<int32_t>> ext(nb);
  int64_t vals = 0, sectors = 0;
  gn::halo_lists(n, rp, ci.data(), part, ext, &vals, &sectors);
  // the halo lists against their definition
  bool lists_ok = true;
  int64_t want_vals = 0, want_sectors = 0;
  for (int b = 0; b < nb; ++b) {
    std::vector<int32_t> x;
    for (int64_t e = rp[part[b]]; e < rp[part[b + 1]]; ++e)
      if (ci[e] < part[b] || ci[e] >= part[b + 1]) x.push_back(ci[e]);
    std::sort(x.begin(), x.end());
    x.erase(std::unique(x.begin(), x.end()), x.end());
    lists_ok = lists_ok && x == ext[b];
    want_vals += (int64_t)x.size();
    for (size_t t = 0; t < x.size(); ++t) want_sectors += (t == 0 || (x[t] >> 3) != (x[t - 1] >> 3));
  }
  CHECK(lists_ok && vals == want_vals && sectors == want_sectors, name);
  gn::HaloBlocks hb;
  gn::encode_halo_blocks(n, rp, ci.data(), part, ext, push, 220 * 1024, &hb);
  CHECK(hb.fits, name);
  if (!hb.fits) return;
  const int R = hb.R, zero_id = R + hb.Lp;
  auto header = [&](int b) { return reinterpret_cast<const gn::HaloHeader*>(hb.blob.get() + hb.hoff[b]); };
  auto at = [&](int b, int off) { return hb.blob.get() + hb.hoff[b] + off; };
  // push: the vertex each inbox slot receives, from the owners' send lists
  std::vector<int32_t> inbox;
  bool pieces_ok = true;
  if (push) {
    inbox.assign((size_t)hb.inbox_slots, -2);  // -2: unwritten, -1: padding
    for (int o = 0; o < nb; ++o) {
      const gn::HaloHeader* H = header(o);
      const int4* pc = reinterpret_cast<const int4*>(at(o, H->off_piece));
      const uint16_t* src = reinterpret_cast<const uint16_t*>(at(o, H->off_src));
      for (int p = 0; p < H->npiece; ++p) {
        const int4 q = pc[p];
        pieces_ok = pieces_ok && q.x % 4 == 0 && q.y % 4 == 0 && q.z % 4 == 0 && q.y > 0 && q.y <= gn::kSendPiece &&
                    q.x + q.y <= hb.inbox_slots;
        if (!pieces_ok) break;
        for (int k = 0; k < q.y; ++k) {
          const int sv = src[q.z + k];
          const bool pad = sv >= zero_id && sv < zero_id + 32;
          pieces_ok = pieces_ok && inbox[q.x + k] == -2 && (pad || sv < part[o + 1] - part[o]);
          inbox[q.x + k] = pad ? -1 : part[o] + sv;
        }
      }
    }
    for (int32_t v : inbox) pieces_ok = pieces_ok && v != -2;
    CHECK(pieces_ok, name);
    if (!pieces_ok) return;
  }
  bool rows_ok = true, ids_ok = true, pad_ok = true, interior_ok = true, dep_ok = true, halo_ok = true;
  for (int b = 0; b < nb; ++b) {
    const gn::HaloHeader* H = header(b);
    const int rb = part[b], nr = part[b + 1] - rb;
    // the vertex a local id reads: own row, halo value, or -1 for a zero slot (-3: invalid)
    std::vector<int32_t> halo(H->lx, -1);
    if (push) {
      for (int h = 0; h < H->lx; ++h) halo[h] = inbox[H->inbox_off + h];
    } else {
      const int32_t* x = reinterpret_cast<const int32_t*>(at(b, H->off_x));
      for (int h = 0; h < H->lx; ++h) halo[h] = x[h];
    }
    auto vertex = [&](int id) -> int32_t {
      if (id < nr) return rb + id;
      if (id >= R && id < R + H->lx) return halo[id - R];
      if (id >= zero_id && id < zero_id + 32) return -1;
      return -3;
    };
    // the halo holds exactly the CTA's external neighbours; its owners are the dependency list
    std::vector<int32_t> hv;
    for (int32_t v : halo)
      if (v >= 0) hv.push_back(v);
    std::sort(hv.begin(), hv.end());
    halo_ok = halo_ok && hv == ext[b];
    std::vector<int32_t> owners;
    for (int32_t v : hv) {
      const int o = (int)(std::upper_bound(part.begin(), part.end(), v) - part.begin()) - 1;
      if (owners.empty() || owners.back() != o) owners.push_back(o);
    }
    const int32_t* dep = reinterpret_cast<const int32_t*>(at(b, H->off_dep));
    dep_ok = dep_ok && H->ndep == (int)owners.size() && std::equal(owners.begin(), owners.end(), dep);
    std::vector<int> seen(nr, 0);
    std::vector<std::vector<int32_t>> got(nr);
    const int2* meta = reinterpret_cast<const int2*>(at(b, H->off_meta));
    const short* srow = reinterpret_cast<const short*>(at(b, H->off_srow));
    const uint16_t* sell = reinterpret_cast<const uint16_t*>(at(b, H->off_sell));
    for (int sl = 0; sl < H->ns; ++sl) {
      const int base = meta[sl].x, W = meta[sl].y;
      for (int k = 0; k < W; ++k) {
        uint32_t real_banks = 0, pad_banks = 0;
        for (int l = 0; l < 32; ++l) {
          const int id = sell[base + (k >> 2) * 128 + l * 4 + (k & 3)], r = srow[sl * 32 + l];
          const int32_t v = vertex(id);
          ids_ok = ids_ok && v != -3 && (r >= 0 || v == -1);
          if (v >= 0 && r >= 0) {
            got[r].push_back(v);
            real_banks |= 1u << (id & 31);
            interior_ok = interior_ok && (sl >= H->ns_int || id < nr);
          } else {
            pad_banks |= 1u << (id & 31);
          }
        }
        pad_ok = pad_ok && (real_banks == 0xffffffffu || !(pad_banks & real_banks));
      }
      for (int l = 0; l < 32; ++l)
        if (srow[sl * 32 + l] >= 0) ++seen[srow[sl * 32 + l]];
    }
    const int* hm = reinterpret_cast<const int*>(at(b, H->off_hmeta));
    const int* hc = reinterpret_cast<const int*>(at(b, H->off_hchunk));
    const uint16_t* hl = reinterpret_cast<const uint16_t*>(at(b, H->off_hl));
    for (int h = 0; h < H->nheavy; ++h) {
      const int r = hm[3 * h];
      ++seen[r];
      for (int c = hm[3 * h + 1]; c < hm[3 * h + 1] + hm[3 * h + 2]; ++c)
        for (int k = 0; k < hc[2 * c + 1]; ++k) {
          const int32_t v = vertex(hl[hc[2 * c] + k]);
          ids_ok = ids_ok && v >= 0;
          got[r].push_back(v);
        }
    }
    for (int r = 0; r < nr; ++r) {
      rows_ok = rows_ok && seen[r] == 1;
      std::sort(got[r].begin(), got[r].end());
      ids_ok = ids_ok && std::equal(got[r].begin(), got[r].end(), ci.begin() + rp[rb + r],
                                    ci.begin() + rp[rb + r + 1]) &&
               (int64_t)got[r].size() == rp[rb + r + 1] - rp[rb + r];
    }
  }
  CHECK(rows_ok, name);
  CHECK(ids_ok, name);
  CHECK(pad_ok, name);
  CHECK(interior_ok, name);
  CHECK(dep_ok, name);
  CHECK(halo_ok, name);
}

// A graph whose first slice needs more than 64 colours: CTA 0's rows 0..31 each read the 64
// even-ranked vertices of 128 in CTA 1 and rows 32..63 the odd-ranked ones, so CTA 0's halo holds
// all 128 and the first slice's 2048 entries fall on 16 banks, 128 on each.
static void crowded_graph(int n, std::vector<int32_t>& rp, std::vector<int32_t>& ci) {
  std::vector<std::vector<int32_t>> adj(n);
  const int base = n / 2 + 5;
  for (int r = 0; r < 64; ++r)
    for (int t = r < 32 ? 0 : 1; t < 128; t += 2) {
      adj[r].push_back(base + t);
      adj[base + t].push_back(r);
    }
  rp.assign(n + 1, 0);
  ci.clear();
  for (int i = 0; i < n; ++i) {
    std::sort(adj[i].begin(), adj[i].end());
    ci.insert(ci.end(), adj[i].begin(), adj[i].end());
    rp[i + 1] = (int32_t)ci.size();
  }
}

static void check_all_blocks(std::mt19937& rng) {
  std::vector<int32_t> rp, ci;
  random_graph(rng, 9000, 6, 40, 4, rp, ci);  // local, with hubs: interior slices, dense halos
  check_blocks("blocks, local graph, pull", 9000, rp, ci, 11, false);
  check_blocks("blocks, local graph, push", 9000, rp, ci, 11, true);
  random_graph(rng, 6000, 8, 0, 3, rp, ci);  // random: most edges cut
  check_blocks("blocks, random graph, pull", 6000, rp, ci, 7, false);
  check_blocks("blocks, random graph, push", 6000, rp, ci, 7, true);
  random_graph(rng, 300, 3, 5, 0, rp, ci);  // one slice per CTA, ragged
  check_blocks("blocks, small graph, push", 300, rp, ci, 3, true);
  check_blocks("blocks, small graph, pull", 300, rp, ci, 3, false);
  {  // a shared-memory limit no block fits: nothing is built
    std::vector<int32_t> part = {0, 150, 300};
    std::vector<std::vector<int32_t>> ext(2);
    int64_t vals = 0, sectors = 0;
    gn::halo_lists(300, rp, ci.data(), part, ext, &vals, &sectors);
    for (bool push : {false, true}) {
      gn::HaloBlocks hb;
      gn::encode_halo_blocks(300, rp, ci.data(), part, ext, push, 1024, &hb);
      CHECK(!hb.fits && !hb.blob, "blocks over the shared-memory limit are not built");
    }
  }
  crowded_graph(600, rp, ci);  // more than 64 colours in a slice, folded past the width
  check_blocks("blocks, crowded banks, pull", 600, rp, ci, 2, false);
  check_blocks("blocks, crowded banks, push", 600, rp, ci, 2, true);
}

int main() {
  std::mt19937 rng(20261204);
  check_colouring(rng);
  check_placement(rng);
  check_all_blocks(rng);
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
