// Test driver for the host setup of the sparsifying preconditioner (csrc/host_spp.cpp):
// builds the nested-dissection structure and one pole's multifrontal factor, then replays
// the device triangular-solve algorithm on the host (supernode products with W_f / W_b,
// update rows summed by the ancestor in CSR order; 2D leaves also through their banded
// L/U and halo couplings) and prints x = P^-1 b.
//
// argv[1] (optional): threads for the elimination tree (default 1)
// argv[2] (optional): "maps" -- also replay the device factorisation's schedule
//         (SppFactorMaps: fronts assembled from the maps, partial LU -- written unblocked:
//         the device's panels and trailing updates give every element the same updates in
//         the same order --, L_SS^-1 and U_SS^-1 by columns, the W products) on the host and
//         print "mapsdiff" with the largest differences from the host factor, relative to
//         the largest entry
//         or "tri" -- print "tri host <nonzeros> <entries>" (and "tri maps ..." for the
//         replayed device factorisation): the entries of the zero triangles (above the
//         diagonal of L_SS^-1 in W_f, below the diagonal of U_SS^-1 in W_b) of every node
//         whose solves run through W, and how many of them are not exactly zero; the
//         supernode products skip those triangles
// stdin:  dim m L shift z_re z_im, then n values of V, then n pairs (re, im) of b
// stdout: "dense" then n pairs of x (every node through W), and for 2D "banded" then n
//         pairs of x (leaves through the banded data)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <string>
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

// The device factorisation's steps (k_factor.cu) with the maps, in FP64 on the host.
static bool factor_with_maps(const SppStructure& st, const SppFactorMaps& mp, const SppStencil& sten,
                             const std::vector<double>& V, double pivot_floor, std::vector<cd>& factor,
                             std::vector<cd>& leafv) {
  const int na = (int)st.offsets.size() / 3, NB = SppStructure::NBR;
  std::vector<cd> fronts((size_t)mp.front_size);
  factor.assign((size_t)st.factor_size, cd(0, 0));
  leafv.assign((size_t)st.leaf_size, cd(0, 0));
  for (const auto& lev : st.levels)
    for (int s : lev) {
      const SppNode& nd = st.nodes[s];
      const int ns = nd.ns, nb = nd.nb, nf = ns + nb, kb = ns + nb;
      cd* F = &fronts[mp.foff[s]];
      std::fill(F, F + (size_t)nf * nf, cd(0, 0));
      for (int k = mp.asm_ptr[s]; k < mp.asm_ptr[s + 1]; ++k) {
        const int src = mp.asm_src[k], t = src % na;
        F[mp.asm_pos[k]] = sten.q[t] + sten.qg[t] * (V[mp.nbr[src]] - sten.lmean);
      }
      const int li = mp.leaf_of[s];
      if (li >= 0) {
        const int bw = st.leaf_bw;
        cd* Fbs = &leafv[st.leaf_voff[li]] + (size_t)ns * bw + (size_t)ns * (bw + 1);
        cd* Fsb = Fbs + (size_t)nb * NB;
        const int* bsi = &st.leaf_bs_idx[st.leaf_ioff_bs[li]];
        const int* sbi = &st.leaf_sb_idx[st.leaf_ioff_sb[li]];
        for (int e = 0; e < nb * NB; ++e) Fbs[e] = bsi[e] >= 0 ? F[(size_t)(ns + e / NB) * nf + bsi[e]] : cd(0, 0);
        for (int e = 0; e < ns * NB; ++e) Fsb[e] = sbi[e] >= 0 ? F[(size_t)(e / NB) * nf + ns + sbi[e]] : cd(0, 0);
      }
      for (int c : {mp.child0[s], mp.child1[s]}) {
        if (c < 0) continue;
        const SppNode& cn = st.nodes[c];
        const int nfc = cn.ns + cn.nb;
        const cd* Fc = &fronts[mp.foff[c]];
        const int* em = &mp.emap[cn.boff];
        for (int a = 0; a < cn.nb; ++a)
          for (int b = 0; b < cn.nb; ++b) F[(size_t)em[a] * nf + em[b]] += Fc[(size_t)(cn.ns + a) * nfc + cn.ns + b];
      }
      for (int k = 0; k < ns; ++k) {
        cd* rk = F + (size_t)k * nf;
        double rown = 0;
        for (int j = k; j < nf; ++j) rown = std::max(rown, std::abs(rk[j]));
        cd piv = rk[k];
        const double ap = std::abs(piv);
        if (ap < pivot_floor * rown || ap == 0.0) {
          const double mag = pivot_floor * (rown > 0 ? rown : 1.0);
          piv = ap > 0 ? piv / ap * mag : cd(mag, 0);
          rk[k] = piv;
        }
        const cd ip = 1.0 / piv;
        for (int i = k + 1; i < nf; ++i) {
          cd* ri = F + (size_t)i * nf;
          if (ri[k] == cd(0, 0)) continue;
          const cd l = ri[k] * ip;
          for (int j = k + 1; j < nf; ++j) ri[j] -= l * rk[j];
          ri[k] = l;
        }
      }
      cd* wf = &factor[nd.wf];
      cd* wb = &factor[nd.wb];
      for (int j = 0; j < ns; ++j) {
        wf[(size_t)j * ns + j] = 1.0;
        for (int i = j + 1; i < ns; ++i) {
          cd acc = 0;
          for (int k = j; k < i; ++k) acc += F[(size_t)i * nf + k] * wf[(size_t)k * ns + j];
          wf[(size_t)i * ns + j] = -acc;
        }
        wb[(size_t)j * kb + j] = 1.0 / F[(size_t)j * nf + j];
        for (int i = j - 1; i >= 0; --i) {
          cd acc = 0;
          for (int k = i + 1; k <= j; ++k) acc += F[(size_t)i * nf + k] * wb[(size_t)k * kb + j];
          wb[(size_t)i * kb + j] = -acc * (1.0 / F[(size_t)i * nf + i]);
        }
      }
      for (int r = 0; r < nb; ++r)
        for (int c = 0; c < ns; ++c) {
          cd acc = 0;
          for (int k = 0; k < ns; ++k) acc += F[(size_t)(ns + r) * nf + k] * wf[(size_t)k * ns + c];
          wf[(size_t)(ns + r) * ns + c] = acc;
        }
      for (int r = 0; r < ns; ++r)
        for (int c = 0; c < nb; ++c) {
          cd acc = 0;
          for (int k = 0; k < ns; ++k) acc += wb[(size_t)r * kb + k] * F[(size_t)k * nf + ns + c];
          wb[(size_t)r * kb + ns + c] = -acc;
        }
      if (li >= 0) {
        const int bw = st.leaf_bw;
        cd* Lb = &leafv[st.leaf_voff[li]];
        cd* Ub = Lb + (size_t)ns * bw;
        for (int i = 0; i < ns; ++i) {
          for (int t = 0; t < bw; ++t) Lb[(size_t)i * bw + t] = i - 1 - t >= 0 ? F[(size_t)i * nf + i - 1 - t] : cd(0, 0);
          for (int t = 0; t <= bw; ++t)
            Ub[(size_t)i * (bw + 1) + t] =
                i + t < ns ? (t == 0 ? 1.0 / F[(size_t)i * nf + i] : F[(size_t)i * nf + i + t]) : cd(0, 0);
        }
      }
    }
  return true;
}

// Entries of the zero triangles of the W blocks of every node solved through W (all
// nodes but the banded 2D leaves), and how many are not exactly zero.
static void tri_count(const SppStructure& st, const std::vector<cd>& factor, long* nonzero, long* entries) {
  *nonzero = 0;
  *entries = 0;
  for (size_t id = 0; id < st.nodes.size(); ++id) {
    if (std::binary_search(st.leaf_nodes.begin(), st.leaf_nodes.end(), (int)id)) continue;
    const SppNode& nd = st.nodes[id];
    const int ns = nd.ns, kb = nd.ns + nd.nb;
    const cd* wf = &factor[nd.wf];
    const cd* wb = &factor[nd.wb];
    for (int r = 0; r < ns; ++r)
      for (int k = 0; k < ns; ++k) {
        if (k > r) {
          ++*entries;
          if (wf[(size_t)r * ns + k] != cd(0, 0)) ++*nonzero;
        }
        if (k < r) {
          ++*entries;
          if (wb[(size_t)r * kb + k] != cd(0, 0)) ++*nonzero;
        }
      }
  }
}

static double max_rel_diff(const std::vector<cd>& a, const std::vector<cd>& b) {
  double mx = 0, d = 0;
  for (size_t i = 0; i < a.size(); ++i) {
    mx = std::max(mx, std::abs(b[i]));
    d = std::max(d, std::abs(a[i] - b[i]));
  }
  return mx > 0 ? d / mx : d;
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
  if (argc > 2 && std::string(argv[2]) == "tri") {
    long nz = 0, ne = 0;
    tri_count(st, pp.factor, &nz, &ne);
    printf("tri host %ld %ld\n", nz, ne);
    const SppFactorMaps mp = spp_factor_maps(st);
    if (mp.ok) {
      SppStencil sten;
      std::vector<cd> gh2, fac, lv;
      spp_pole_stencil(st, 2.0 * M_PI * M_PI / (L * L), V.data(), shift, cd(zr, zi), sten, gh2);
      factor_with_maps(st, mp, sten, V, 1e-12, fac, lv);
      tri_count(st, fac, &nz, &ne);
      printf("tri maps %ld %ld\n", nz, ne);
    }
    return 0;
  }
  if (argc > 2 && std::string(argv[2]) == "maps") {
    const SppFactorMaps mp = spp_factor_maps(st);
    if (!mp.ok) {
      printf("mapsdiff unsupported\n");
    } else {
      SppStencil sten;
      std::vector<cd> gh2, fac, lv;
      spp_pole_stencil(st, 2.0 * M_PI * M_PI / (L * L), V.data(), shift, cd(zr, zi), sten, gh2);
      factor_with_maps(st, mp, sten, V, 1e-12, fac, lv);
      printf("mapsdiff %.3e %.3e\n", max_rel_diff(fac, pp.factor), lv.empty() ? 0.0 : max_rel_diff(lv, pp.leafval));
    }
  }
  for (int mode = 0; mode < (st.leaf_nodes.empty() ? 1 : 2); ++mode) {
    printf("%s\n", mode ? "banded" : "dense");
    for (const cd& v : replay(st, pp, b, mode == 1)) printf("%.17g %.17g\n", v.real(), v.imag());
  }
  return 0;
}
