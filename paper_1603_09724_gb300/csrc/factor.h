// Device-side multifrontal factorisation of the sparsifying matrix P (k_factor.cu).
#pragma once
#include <cuda_runtime.h>

namespace omm {

// Device arrays of the structure (SppStructure, SppFactorMaps) and the per-pole stencil
// data; every pointer is device memory.
struct FactorArgs {
  const int* node_ns;
  const int* node_nb;
  const int* node_boff;
  const long long* node_wf;
  const long long* node_wb;
  const long long* foff;       // front offset per node (entries, within a pole's workspace)
  const int* child0;
  const int* child1;
  const int* asm_ptr;          // per node: range of its P entries
  const int* asm_pos;          // front position (row * nf + col)
  const int* asm_src;          // natural row * na + stencil index
  const int* nbr;              // n * na stencil neighbours (natural)
  const int* emap;             // per boundary entry: position in the parent's front
  const int* leaf_of;          // per node: banded leaf index or -1
  const long long* leaf_voff;
  const int* leaf_ioff_bs;
  const int* leaf_ioff_sb;
  const int* leaf_bs_idx;
  const int* leaf_sb_idx;
  int leaf_bw;
  int na;                      // stencil size
  int nnodes;
  long long front_size;        // front entries per pole
  long long factor_size;       // factor entries per pole
  long long leaf_size;         // leaf entries per pole
  const double* V;             // n potential values
  double lmean;                // l = <V>
  const double2* q;            // P x na: q of each pole
  const double2* qg;           // P x na: (qG)(0, a) of each pole
  double pivot_floor;
};

// The launch shape of one tree height (computed on the host from the node sizes).
struct FactorHeight {
  static constexpr int kMaxPanels = 64;   // panels of 32 pivots: ns up to 2048
  const int* nodes = nullptr;   // device: node ids of the height
  int count = 0;                // nodes
  int max_ns = 0;               // largest ns of the height
  int max_nf = 0;               // largest front (ns + nb) of the height
  int npanels = 0;              // ceil(max_ns / 32)
  int trail_tiles[kMaxPanels];  // per panel: largest count of 32 x 32 trailing-update tiles
  bool has_leaves = false;      // some node of the height is a banded 2D leaf
  bool dense_nodes = false;     // some node of the height needs its dense W blocks
  int wprod_tiles = 0;          // largest count of 32 x 32 output tiles of the W products
};

// One tree height of the factorisation for P poles, in FP64: the nodes of hh, all of whose
// children were factorised by earlier calls.  fronts: P x front_size work space;
// factor / leafv: P x factor_size W blocks and P x leaf_size banded leaf data, written for
// these nodes (a 2D leaf's W blocks are left as they are: the solves use its banded data);
// pstats: P x nnodes x 3 doubles (smallest and largest pivot magnitude, pivots raised).
// Errors: cudaErrorInvalidValue for P or count outside [1, 65535] or npanels above
// kMaxPanels.
cudaError_t launch_factor_height(const FactorArgs& f, const FactorHeight& hh, int P, double2* fronts,
                                 double2* factor, double2* leafv, double* pstats, cudaStream_t st);

// dst[i] = src[i] rounded to complex64 (a mixed handle's factor and leaf data).
cudaError_t launch_factor_to_c64(const double2* src, float2* dst, size_t count, cudaStream_t st);

}  // namespace omm
