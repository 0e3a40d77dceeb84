// Host-side setup of the sparsifying preconditioner (Sec. 3.2): the stencil row q of
// eq. QG, the sparse matrix P of eq. P, a nested-dissection ordering of the periodic
// grid and the multifrontal LU factorisation of P (dense supernodes), laid out for the
// device triangular solves.
#pragma once
#include <complex>
#include <cstdint>
#include <vector>

namespace omm {

using cd = std::complex<double>;

struct SppNode {
  int off;      // first ND index of the supernode's unknowns
  int ns;       // number of unknowns (separator or leaf box)
  int nb;       // boundary size |B(s)| (ancestor unknowns coupled to the subtree)
  int boff;     // offset into SppStructure::bnat / bnd
  int uoff;     // first row of this node's update vector in the u buffer
  long long wf;  // offset of W_f = [L_SS^-1 ; L_BS L_SS^-1] ((ns + nb) x ns, row-major) in a pole's factor
  long long wb;  // offset of W_b = [U_SS^-1 , -U_SS^-1 U_SB] (ns x (ns + nb), row-major)
  int parent;   // parent node (-1 at the root)
  int height;   // 0 for leaves
};

struct SppStructure {
  int dim = 0, m = 0, r = 1;
  int n = 0;
  std::vector<int> perm;      // perm[nd] = natural index of ND unknown nd
  std::vector<int> iperm;     // iperm[natural] = ND index
  std::vector<SppNode> nodes; // postorder
  std::vector<int> bnat;      // boundary unknowns (natural indices), per node
  std::vector<int> bnd;       // same, ND indices (sorted ascending per node)
  std::vector<std::vector<int>> levels;  // node ids per height
  std::vector<int> contrib_ptr;  // CSR over ND rows: contributions u-row indices
  std::vector<int> contrib_idx;
  int urows = 0;               // total rows of update vectors
  long long factor_size = 0;   // complex entries per pole
  int max_ns = 0, max_nb = 0;
  std::vector<int> offsets;    // stencil offsets, flattened (dx, dy, dz) triples, x fastest
  // row blocks of RB rows per level for the device products: (node, first row) pairs
  static constexpr int RB = 64;
  std::vector<int> fblocks, bblocks;
  std::vector<int> fstart, fcount, bstart, bcount;
  std::vector<int> fkmax, bkmax;   // per level: largest K of the forward / backward products
  // leaves (height 0, no children): banded L, U and the original sparse coupling to the halo
  int leaf_bw = 0;                 // bandwidth of the leaf LU in the leaf's own (x-fastest) order
  static constexpr int NBR = 9;    // max couplings of one unknown (the 3^2 stencil)
  std::vector<int> leaf_nodes;     // node ids of the leaves
  std::vector<long long> leaf_voff;// per leaf: offset of its values in a pole's leaf array
  std::vector<int> leaf_ioff_bs;   // per leaf: offset into leaf_bs_idx (nb * NBR)
  std::vector<int> leaf_ioff_sb;   // per leaf: offset into leaf_sb_idx (ns * NBR)
  std::vector<int> leaf_bs_idx;    // halo row j -> leaf columns i coupled by P (or -1)
  std::vector<int> leaf_sb_idx;    // leaf row i -> halo columns j coupled by P (or -1)
  long long leaf_size = 0;         // complex values per pole: per leaf L band (ns*bw),
                                   // U band with inverted diagonal (ns*(bw+1)), F_BS (nb*NBR), F_SB (ns*NBR)
};

struct SppPole {
  std::vector<cd> q;            // stencil row (|a| entries, same order as offsets)
  std::vector<cd> factor;       // per node W_f and W_b (see SppNode)
  std::vector<cd> leafval;      // per leaf banded factors and couplings (see SppStructure)
  double pivot_min = 0, pivot_max = 0;
  int nperturbed = 0;
  double sigma_min = 0, sigma_max = 0;   // singular values of G(a, a^c)
};

// The stencil data of one pole (eqs. GLu, QG, P): q, (qG)(0, a) and the mean potential l,
// so that P(j, j + o_t) = q_t + qg_t (V_{j+o_t} - l).
struct SppStencil {
  std::vector<cd> q, qg;
  double lmean = 0;
  double sigma_min = 0, sigma_max = 0;   // singular values of G(a, a^c)
};

// Index maps of a multifrontal factorisation on the device, built once per structure.
// Node s owns an nf x nf front (nf = ns + nb, row-major, unknowns then boundary) at
// foff[s] in a pole's front workspace; its P entries are asm_pos / asm_src over
// [asm_ptr[s], asm_ptr[s + 1]) (front position, natural row * na + stencil index t);
// after the partial LU its trailing nb x nb block is the update matrix, which the parent
// adds at the rows / columns emap[boff + a] of its own front.  ok is false when a front
// position would receive two entries of P (grids too small for the stencil) or the tree
// is not binary; the host factorisation then stays in use.
struct SppFactorMaps {
  std::vector<long long> foff;
  long long front_size = 0;        // entries per pole
  std::vector<int> child0, child1; // children in the host's order, -1 if none
  std::vector<int> asm_ptr, asm_pos, asm_src;
  std::vector<int> nbr;            // n * na: natural index of the stencil neighbour j + o_t
  std::vector<int> emap;           // per boundary entry (layout of bnd)
  std::vector<int> leaf_of;        // per node: its index among the banded leaves, or -1
  bool ok = false;
};

// Builds the ND structure for an m^dim periodic grid and stencil radius r.
SppStructure spp_build_structure(int dim, int m, int r);

// The device factorisation's maps for a structure.
SppFactorMaps spp_factor_maps(const SppStructure& st);

// q, (qG)(0, a), l and the Green symbol of one pole (the part of spp_setup_pole before
// the factorisation); ghat_out as for spp_setup_pole.
void spp_pole_stencil(const SppStructure& st, double kin, const double* V, double shift, cd z, SppStencil& out,
                      std::vector<cd>& ghat_out);

// Per pole: q by the SVD of G(a, a^c), P assembly, multifrontal LU with static pivoting.
// kin: (2 pi^2 / L^2); V: n reals; shift: sigma; z: pole.  ghat_out (n) receives
// 1/(T(k) + l - sigma - z) / n (the Green symbol with the inverse-DFT scale folded in).
// threads: workers for the supernodes of this pole's elimination tree (1 = sequential);
// the factor is bitwise the same for any value.
void spp_setup_pole(const SppStructure& st, double kin, const double* V, double shift, cd z, double pivot_floor,
                    SppPole& out, std::vector<cd>& ghat_out, int threads = 1);

// Green symbol only (for the kinetic inner preconditioner).
void green_symbol(int dim, int m, double kin, double lmean, double shift, cd z, std::vector<cd>& ghat_out);

}  // namespace omm
