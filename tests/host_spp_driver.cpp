// Test driver for the host setup of the sparsifying preconditioner (csrc/host_spp.cpp):
// builds the nested-dissection structure and one pole's multifrontal factor, then replays
// the device triangular-solve algorithm on the host (supernode products with W_f / W_b,
// update rows summed by the ancestor in CSR order; 2D leaves also through their banded
// L/U and halo couplings) and prints x = P^-1 b.
//
// argv[1] (optional): threads for the elimination tree (default 1)
// stdin:  dim m L shift z_re z_im, then n values of V, then n pairs (re, im) of b
// stdout: "dense" then n pairs of x (every node through W), and for 2D "banded" then n
//         pairs of x (leaves through the banded data)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "spp.h"

using namespace omm;

static std::vector<cd> replay(const SppStructure& st, const SppPole& pp, const std::vector<cd>& b, bool banded) {
  const int n = st.n, NB = SppStructure::NBR;
  std::vector<cd> ynd(n), x(n), u(st.urows);
  auto leaf_index = [&](int id) -> long {
    if (!banded) return -1;
    auto it = std::lower_bound(st.leaf_nodes.begin(), st.leaf_nodes.end(), id);
    return (it != st.leaf_nodes.end() && *it == id) ? (long)(it - st.leaf_nodes.begin()) : -1;
  };
  for (size_t h = 0; h < st.levels.size(); ++h)
    for (int id : st.levels[h]) {
      const SppNode& nd = st.nodes[id];
      const int ns = nd.ns, nb = nd.nb;
      std::vector<cd> B(ns);
      for (int i = 0; i < ns; ++i) {
        B[i] = b[st.perm[nd.off + i]];
        for (int e = st.contrib_ptr[nd.off + i]; e < st.contrib_ptr[nd.off + i + 1]; ++e) B[i] -= u[st.contrib_idx[e]];
      }
      const long li = leaf_index(id);
      if (li >= 0) {
        const int bw = st.leaf_bw;
        const cd* Lb = &pp.leafval[st.leaf_voff[li]];
        const cd* Ub = Lb + (size_t)ns * bw;
        const cd* Fbs = Ub + (size_t)ns * (bw + 1);
        for (int i = 0; i < ns; ++i)
          for (int t = 0; t < bw && i - 1 - t >= 0; ++t) B[i] -= Lb[(size_t)i * bw + t] * B[i - 1 - t];
        for (int i = 0; i < ns; ++i) ynd[nd.off + i] = B[i];
        for (int i = ns - 1; i >= 0; --i) {
          cd acc = B[i];
          for (int t = 1; t <= bw && i + t < ns; ++t) acc -= Ub[(size_t)i * (bw + 1) + t] * B[i + t];
          B[i] = Ub[(size_t)i * (bw + 1)] * acc;
        }
        const int* bsi = &st.leaf_bs_idx[st.leaf_ioff_bs[li]];
        for (int j = 0; j < nb; ++j) {
          cd acc = 0;
          for (int t = 0; t < NB; ++t)
            if (bsi[j * NB + t] >= 0) acc += Fbs[(size_t)j * NB + t] * B[bsi[j * NB + t]];
          u[nd.uoff + j] = acc;
        }
      } else {
        const cd* W = &pp.factor[nd.wf];
        for (int r = 0; r < ns + nb; ++r) {
          cd acc = 0;
          for (int k = 0; k < ns; ++k) acc += W[(size_t)r * ns + k] * B[k];
          if (r < ns) ynd[nd.off + r] = acc; else u[nd.uoff + r - ns] = acc;
        }
      }
    }
  for (int h = (int)st.levels.size() - 1; h >= 0; --h)
    for (int id : st.levels[h]) {
      const SppNode& nd = st.nodes[id];
      const int ns = nd.ns, nb = nd.nb;
      const long li = leaf_index(id);
      if (li >= 0) {
        const int bw = st.leaf_bw;
        const cd* Lb = &pp.leafval[st.leaf_voff[li]];
        const cd* Ub = Lb + (size_t)ns * bw;
        const cd* Fsb = Ub + (size_t)ns * (bw + 1) + (size_t)nb * NB;
        const int* sbi = &st.leaf_sb_idx[st.leaf_ioff_sb[li]];
        std::vector<cd> y(ns);
        for (int i = 0; i < ns; ++i) {
          cd acc = 0;
          for (int t = 0; t < NB; ++t)
            if (sbi[i * NB + t] >= 0) acc += Fsb[(size_t)i * NB + t] * x[st.bnat[nd.boff + sbi[i * NB + t]]];
          y[i] = acc;
        }
        for (int i = 0; i < ns; ++i)
          for (int t = 0; t < bw && i - 1 - t >= 0; ++t) y[i] -= Lb[(size_t)i * bw + t] * y[i - 1 - t];
        for (int i = 0; i < ns; ++i) y[i] = ynd[nd.off + i] - y[i];
        for (int i = ns - 1; i >= 0; --i) {
          cd acc = y[i];
          for (int t = 1; t <= bw && i + t < ns; ++t) acc -= Ub[(size_t)i * (bw + 1) + t] * y[i + t];
          y[i] = Ub[(size_t)i * (bw + 1)] * acc;
        }
        for (int i = 0; i < ns; ++i) x[st.perm[nd.off + i]] = y[i];
      } else {
        const cd* W = &pp.factor[nd.wb];
        const int K = ns + nb;
        std::vector<cd> B(K);
        for (int i = 0; i < ns; ++i) B[i] = ynd[nd.off + i];
        for (int j = 0; j < nb; ++j) B[ns + j] = x[st.bnat[nd.boff + j]];
        for (int r = 0; r < ns; ++r) {
          cd acc = 0;
          for (int k = 0; k < K; ++k) acc += W[(size_t)r * K + k] * B[k];
          x[st.perm[nd.off + r]] = acc;
        }
      }
    }
  return x;
}

int main(int argc, char** argv) {
  const int threads = argc > 1 ? std::atoi(argv[1]) : 1;
  int dim, m;
  double L, shift, zr, zi;
  if (scanf("%d %d %lf %lf %lf %lf", &dim, &m, &L, &shift, &zr, &zi) != 6) return 2;
  const SppStructure st = spp_build_structure(dim, m, 1);
  const int n = st.n;
  std::vector<double> V(n);
  for (auto& v : V)
    if (scanf("%lf", &v) != 1) return 2;
  std::vector<cd> b(n);
  for (auto& v : b) {
    double re, im;
    if (scanf("%lf %lf", &re, &im) != 2) return 2;
    v = cd(re, im);
  }
  SppPole pp;
  std::vector<cd> gh;
  spp_setup_pole(st, 2.0 * M_PI * M_PI / (L * L), V.data(), shift, cd(zr, zi), 1e-12, pp, gh, threads);
  for (int mode = 0; mode < (st.leaf_nodes.empty() ? 1 : 2); ++mode) {
    printf("%s\n", mode ? "banded" : "dense");
    for (const cd& v : replay(st, pp, b, mode == 1)) printf("%.17g %.17g\n", v.real(), v.imag());
  }
  return 0;
}
