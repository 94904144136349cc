// Device view of the Morse excluded-volume state (neighbour lists with a
// skin over a cell list; the kernels are in morse.cu).
#pragma once
#include "common.cuh"

namespace ibm {

struct MorseDev {
  float D0, alpha, r0, rc2;
  float rl2;          // (rc + skin)^2: neighbour-list cutoff
  float half_skin2;   // (skin / 2)^2: a larger move since the last build triggers a rebuild
  int cap;            // neighbour-list entries per marker
  int nb[3];          // bins per axis (each at least rc + skin wide)
  float inv_bs[3];    // 1 / bin size
  int n_bins;
  int* count;         // [n_bins] markers per bin (zero between steps)
  int* start;         // [n_bins + 1] exclusive prefix of count
  int* block_sum;     // [scan blocks]
  int* bin_of;        // [M]
  int* rank;          // [M] position within the bin
  float4* sorted;     // [M] wrapped position, owner body (int bits in w), by bin
  int* sorted_id;     // [M] marker of each sorted slot
  int* bin_owner;     // [n_bins] the one body all markers of a bin belong to, -2 if several, -1 if empty
  const int* owner;   // [M] body of a participating marker, -1 otherwise
  float4* ref;        // [M] unwrapped position at the last list build
  float4* cur;        // [M] wrapped position and owner (int bits in w), this step
  int* n_nbr;         // [M] list length
  int* nbr;           // [M][cap] markers of other bodies within rc + skin at the last build
  int* flags;         // [0] rebuild this step, [1] a list overflowed at the last build
};

}  // namespace ibm
