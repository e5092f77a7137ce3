// Accumulator layout of the slot-wise scatter (host setup and kernels).
//
// A warp sums one CSR row (or the three rows of a node) in shared memory, one
// 8-byte FP32 pair per nonzero. The lanes of one slot (one cell around the
// DOF) touch the entries of that cell's columns, local column m on lane
// m mod 32, and shared memory serves a half-warp's 8-byte accesses in one
// wavefront only when its 16 entries lie in distinct bank pairs (entry mod 16).
//
// Q1 elasticity (24 local DOFs, comp-major: m = 8 c + a): a node row has the
// 27 neighbour nodes x + 3y + 9z (x, y, z in 0..2) times 3 components as its
// nonzeros, k = 3 (x + 3y + 9z) + c, and a cell around the node touches one
// 2 x 2 x 2 block of them. Stored in nonzero order, the comp 0 and comp 1
// entries of that block (lanes 0..15) share bank pairs, about 1.8 wavefronts
// per half-warp. The map below gives each entry the bank pair
//   comp 0: beta,  comp 1: 8 + beta,  comp 2: 8 + (beta ^ 7),
// beta = (x & 1) | (y & 1) << 1 | (z & 1) << 2, which differs for the eight
// nodes of any 2 x 2 x 2 block; lanes 0..15 (comps 0 and 1) then fill all 16
// bank pairs, and lanes 16..23 (comp 2) use 8..15, leaving bank pair 0 to the
// dummy entry of the padding lanes 24..31. Within a bank pair the entry's row
// is the node's rank among the nodes of its parity class (x >> 1 | y >> 1 << 1
// | z >> 1 << 2; comp 2 counts down from 8, and the two classes that share a
// bank pair have disjoint ranks), so entries run to 143. The map is
// one-to-one for every k; it is conflict-free for rows whose columns are the
// 27 neighbours in lexicographic order (the interior nodes of a structured
// mesh numbered by list_dofs, most rows) and worse than nonzero order on the
// others, so the host applies it only to the rows whose slots it serves in
// fewer wavefronts, and marks them with bit 14 of every position (bit 15 is
// the first-contribution flag; entries stay below 2^14). Rows with more than
// 81 nonzeros (unstructured meshes) continue after entry 143.
#pragma once

#if defined(__CUDACC__)
#define FE_HD __host__ __device__ __forceinline__
#else
#define FE_HD inline
#endif

namespace feasm {

constexpr int kQ1eEntries = 144;  // entries of the map for k < 81

FE_HD int q1e_entry(int k) {
  if (k >= 81) return k + (kQ1eEntries - 81);
  const int r = k / 3, c = k - 3 * r;
  const int z = r / 9, y = (r - 9 * z) / 3, x = r - 9 * z - 3 * y;
  const int beta = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2);
  const int rank = (x >> 1) | ((y >> 1) << 1) | ((z >> 1) << 2);
  if (c == 0) return beta + 16 * rank;
  if (c == 1) return 8 + beta + 16 * rank;
  return 8 + (beta ^ 7) + 16 * (8 - rank);
}

constexpr int kPosEntry = 0x3fff;    // position bits: the accumulator entry
constexpr int kPosMapped = 0x4000;   // position bit: the row's entries follow q1e_entry
constexpr int kPosFirst = 0x8000;    // position bit: first contribution of its nonzero

// Entry of the k-th nonzero of a row (mapped: the Q1 elasticity map).
FE_HD int slot_entry(bool mapped, int k) { return mapped ? q1e_entry(k) : k; }

// Entries per row before the row's dummy entry (a multiple of 16, so that the
// dummy lies in bank pair 0).
inline int slot_acc_stride(int nl, long long max_row_nnz) {
  const long long n = nl == 24 ? (max_row_nnz <= 81 ? kQ1eEntries : max_row_nnz + (kQ1eEntries - 81)) : max_row_nnz;
  return int((n + 15) & ~15LL);
}

}  // namespace feasm
