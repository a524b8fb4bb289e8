// Host-side checks of the halo block builder's slice colouring and send-piece placement
// (gn_halo_build.cu, included here for its file-local functions), linked against libgn.so for
// the rest.  The placement is compared slot for slot with its rule written out plainly.  No GPU is used.  Prints "ok" and returns 0 when every check passes; prints what
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

int main() {
  std::mt19937 rng(20261204);
  check_colouring(rng);
  check_placement(rng);
  if (failures) {
    std::printf("%d failures\n", failures);
    return 1;
  }
  std::printf("ok\n");
  return 0;
}
