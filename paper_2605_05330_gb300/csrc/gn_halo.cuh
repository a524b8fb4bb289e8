// gn_halo.cuh -- the packed per-CTA block of the halo gather mode, shared by the kernel
// (gn_halo.cu) and the host code that builds the blocks (gn_halo_build.cu).
#pragma once

#include <stdint.h>

namespace gn {

// Version of what the builder writes into the blocks (layout and contents for a given graph and
// partition).  It changes with every change to gn_halo_build.cu that changes its output, so the
// recorded DRAM traffic of the kernel, which depends on it, is tied to this header and not to
// the builder's code.
constexpr int kHaloLayoutVersion = 4;

// header of a CTA block (int32 words), followed by 16-byte aligned sections
struct HaloHeader {
  int ns_int;      // interior slices (every row's neighbours are own rows)
  int ns;          // all slices
  int nheavy;      // heavy rows
  int lx;          // external halo length (push: inbox slots, each owner's run padded to 4)
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
  int off_piece;   // int4 per piece: (first inbox slot, length, first source, 0), multiples of 4
  int off_src;     // uint16 per sent slot: the own row it comes from (padding: a zero slot)
  int off_x;       // pull: int32 per halo value, its vertex id
  int pad0;
};

constexpr int kHeavyHalo = 64;    // rows with more entries are cut into chunks
constexpr int kHeavyChunk = 256;  // entries per chunk (8 per lane)
constexpr int kSendPiece = 128;   // inbox slots per send piece

}  // namespace gn
