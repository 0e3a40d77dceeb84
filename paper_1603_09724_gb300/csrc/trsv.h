// Device-side description of the nested-dissection multifrontal factor structure.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <vector>

namespace omm {

struct TrsvArgs {
  // per node (device arrays)
  const int* node_ns;
  const int* node_nb;
  const int* node_off;
  const int* node_boff;
  const int* node_uoff;
  const long long* node_wf;   // W_f offset ((ns + nb) x ns, row-major)
  const long long* node_wb;   // W_b offset (ns x (ns + nb), row-major)
  const int* perm;            // ND -> natural
  const int* bnat;            // boundary natural indices
  const int* bnd;             // the same boundary unknowns, ND indices
  const int* contrib_ptr;     // n + 1
  const int* contrib_idx;
  long long factor_size;      // complex entries per pole
  size_t n;                   // grid points
  int N;                      // right-hand sides per pole
  size_t S;                   // total systems (rows stride of the u buffer)
};

struct TrsvLevels {
  int nlevels;
  const int* fblocks;         // device: (node, first row) pairs, forward products, by height
  const int* bblocks;         // device: same for the backward products
  std::vector<int> fstart, fcount, bstart, bcount;   // host, per height
  std::vector<int> fkmax, bkmax;                      // host, per height: shared-memory sizing
  const int* lunk;            // device: ND indices of the unknowns of each height, concatenated
  std::vector<int> ustart, ucount;                    // host, per height: range in lunk
};

// Leaves: banded L and U (inverted diagonal) of the leaf front and its original sparse
// coupling to the halo, per pole in one array (see SppStructure).
struct LeafArgs {
  int nleaves = 0;
  int bw = 0;
  int max_ns = 0;
  int max_nb = 0;
  const int* nodes = nullptr;
  const long long* voff = nullptr;
  const int* ioff_bs = nullptr;
  const int* ioff_sb = nullptr;
  const int* bs_idx = nullptr;
  const int* sb_idx = nullptr;
  long long leaf_size = 0;
  const void* vals = nullptr;   // P * leaf_size complex values
};

size_t trsv_smem_bytes(bool dbl, int max_ns, int max_nb);
// b (ND order, S systems) -> x (natural order); ynd, u, xnd (ND order) work buffers, each
// S x n except u (urows x S).  factor: P poles' blocks.
// phases: bit 0 leaves forward, bit 1 levels forward, bit 2 levels backward, bit 3 leaves
// backward (SPP_ALL = 15); the phases must run in that order.  overlap: every launch is a
// programmatic dependent launch, whose prologue (factor values, index lists) runs while
// the launch before it on the stream finishes.
constexpr int SPP_LEAF_FWD = 1, SPP_LEVELS_FWD = 2, SPP_LEVELS_BWD = 4, SPP_LEAF_BWD = 8, SPP_ALL = 15;
cudaError_t launch_spp_solve(int phases, bool dbl, const TrsvArgs& a, const TrsvLevels& lv, const LeafArgs& la, int P,
                             const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                             const int* active, size_t smem, bool overlap, cudaStream_t st);

// All supernode heights (leaves excluded when `leaves`) of one application, every pole of
// the launch, in one cooperative launch with grid barriers between the phases; bar: 3
// unsigned on the device (arrival count, generation, error flag: set when a bounded
// barrier wait gave up), zero before the first launch.  *done is false when the
// structure does not fit the persistent kernel (the caller then launches per height).
cudaError_t launch_spp_levels_persistent(bool dbl, const TrsvArgs& a, const TrsvLevels& lv, bool leaves, int P,
                                         const void* b, void* ynd, void* u, void* x, void* xnd, const void* factor,
                                         const int* active, unsigned* bar, cudaStream_t st, bool* done);

}  // namespace omm
