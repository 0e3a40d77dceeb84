// Sparsifying preconditioner setup on the host in FP64 (Sec. 3.2).
//
//   G = (T + l - sigma - z)^-1 with l = <V> (eq. GLu), a circulant: G(i, j) = g[i - j]
//   Q(j, a(j)) = q for every j: q = conj(u_min), u_min the left singular vector of
//     G(a, a^c) for its smallest singular value (Householder QR of G(a, a^c)^*, then a
//     one-sided Jacobi SVD of its R) (eq. QG)
//   P_{j, j+o} = q_o + (qG)_o (V_{j+o} - l) on the stencil, 0 elsewhere (eq. P)
//   P = L U by nested dissection (recursive bisection of the periodic grid by grid
//   lines / planes) and a multifrontal factorisation with dense fronts, no pivoting
//   (pivots below pivot_floor * row size are raised and counted).
#include <algorithm>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <mutex>
#include <thread>

#include "spp.h"

namespace omm {

namespace {

const double kPi = 3.14159265358979323846264338327950288;

inline int wrap(int a, int m) { a %= m; return a < 0 ? a + m : a; }

struct Box {
  int lo[3], ext[3];
  bool per[3];
};

struct Builder {
  int dim, m, r;
  SppStructure* st;
  std::vector<std::vector<int>> node_pts;   // natural indices per node
  std::vector<Box> node_box;
  std::vector<int> node_children_a, node_children_b;

  int flat(int x, int y, int z) const { return x + m * (y + m * z); }

  void points(const Box& b, std::vector<int>& out) const {
    const int ez = dim == 3 ? b.ext[2] : 1;
    for (int tz = 0; tz < ez; ++tz)
      for (int ty = 0; ty < b.ext[1]; ++ty)
        for (int tx = 0; tx < b.ext[0]; ++tx)
          out.push_back(flat(wrap(b.lo[0] + tx, m), wrap(b.lo[1] + ty, m), dim == 3 ? wrap(b.lo[2] + tz, m) : 0));
  }

  int add_node(std::vector<int>&& pts, const Box& b, int ca, int cb) {
    node_pts.push_back(std::move(pts));
    node_box.push_back(b);
    node_children_a.push_back(ca);
    node_children_b.push_back(cb);
    return (int)node_pts.size() - 1;
  }

  int nd(const Box& b) {
    bool anyper = false;
    int maxext = 0;
    for (int d = 0; d < dim; ++d) {
      if (b.per[d]) anyper = true;
      maxext = std::max(maxext, b.ext[d]);
    }
    for (int d = 0; d < dim; ++d)
      if (b.ext[d] <= 0) return -1;
    const int leaf_ext = (dim == 3) ? 4 : 8;
    if (!anyper && maxext <= leaf_ext) {
      std::vector<int> pts;
      points(b, pts);
      return add_node(std::move(pts), b, -1, -1);
    }
    // cut dimension: a periodic one first (largest), else the largest extent >= 3
    int cd = -1;
    for (int d = 0; d < dim; ++d)
      if (b.per[d] && (cd < 0 || b.ext[d] > b.ext[cd])) cd = d;
    if (cd < 0)
      for (int d = 0; d < dim; ++d)
        if (b.ext[d] >= 3 && (cd < 0 || b.ext[d] > b.ext[cd])) cd = d;
    if (cd < 0) {
      std::vector<int> pts;
      points(b, pts);
      return add_node(std::move(pts), b, -1, -1);
    }
    Box c1 = b, c2 = b, s1 = b, s2 = b;
    std::vector<int> sep;
    if (b.per[cd]) {
      const int h = m / 2;
      c1.per[cd] = c2.per[cd] = false;
      c1.lo[cd] = 1; c1.ext[cd] = h - 1;
      c2.lo[cd] = h + 1; c2.ext[cd] = m - h - 1;
      s1.per[cd] = s2.per[cd] = false;
      s1.lo[cd] = 0; s1.ext[cd] = 1;
      s2.lo[cd] = h; s2.ext[cd] = 1;
      const int a = nd(c1);
      const int bb = nd(c2);
      points(s1, sep);
      points(s2, sep);
      return add_node(std::move(sep), b, a, bb);
    }
    const int mid = b.lo[cd] + b.ext[cd] / 2;
    c1.ext[cd] = mid - b.lo[cd];
    c2.lo[cd] = mid + 1;
    c2.ext[cd] = b.lo[cd] + b.ext[cd] - mid - 1;
    s1.lo[cd] = mid; s1.ext[cd] = 1;
    const int a = nd(c1);
    const int bb = nd(c2);
    points(s1, sep);
    return add_node(std::move(sep), b, a, bb);
  }

  // unknowns coupled to box b through fill: points outside b within distance r (per
  // non-periodic dimension; periodic dimensions are covered by the box)
  void halo(const Box& b, std::vector<int>& out) const {
    int lo[3], ext[3];
    for (int d = 0; d < 3; ++d) {
      if (d >= dim) { lo[d] = 0; ext[d] = 1; continue; }
      if (b.per[d]) { lo[d] = 0; ext[d] = m; }
      else { lo[d] = b.lo[d] - r; ext[d] = std::min(m, b.ext[d] + 2 * r); }
    }
    // membership by stamps in one array over the grid: points of b get stamp_in, points
    // already emitted stamp_seen (fresh values per call, so earlier calls' marks never match)
    if (mark.empty()) mark.assign((size_t)st->n, 0);
    const int stamp_in = ++stamp, stamp_seen = ++stamp;
    {
      std::vector<int> pts;
      points(b, pts);
      for (int p : pts) mark[p] = stamp_in;
    }
    for (int tz = 0; tz < ext[2]; ++tz)
      for (int ty = 0; ty < ext[1]; ++ty)
        for (int tx = 0; tx < ext[0]; ++tx) {
          const int p = flat(wrap(lo[0] + tx, m), wrap(lo[1] + ty, m), dim == 3 ? wrap(lo[2] + tz, m) : 0);
          if (mark[p] == stamp_in || mark[p] == stamp_seen) continue;
          mark[p] = stamp_seen;
          out.push_back(p);
        }
  }
  mutable std::vector<int> mark;   // halo(): per grid point, the stamp of its last visit
  mutable int stamp = 0;
};

// out[x] = sum_k in[k * istride] W^{k x} for x < len, W = e^{+2 pi i / len}, by decimation in
// time over the smallest prime factor r of len: r transforms of length len / r over the
// residues k = s (mod r), then X[k + q t] = sum_s W^{s (k + q t)} Y_s[k] (q = len / r).  A
// prime length is one direct sum.  w[j] = e^{+2 pi i j / M} with M = len * wstep.
void dft_plus(const cd* in, int istride, cd* out, int len, const cd* w, int wstep, int M) {
  if (len == 1) {
    out[0] = in[0];
    return;
  }
  int r = len;
  for (int f = 2; f * f <= len; ++f)
    if (len % f == 0) {
      r = f;
      break;
    }
  const int q = len / r;
  for (int s = 0; s < r; ++s) dft_plus(in + (size_t)s * istride, istride * r, out + (size_t)s * q, q, w, wstep * r, M);
  cd ys[8];
  std::vector<cd> yv;
  cd* y = ys;
  if (r > 8) {
    yv.resize(r);
    y = yv.data();
  }
  for (int k = 0; k < q; ++k) {
    for (int s = 0; s < r; ++s) y[s] = out[(size_t)s * q + k];
    for (int t = 0; t < r; ++t) {
      const int x = k + q * t;
      double re = 0.0, im = 0.0;
      int e = 0;   // s x mod len
      for (int s = 0; s < r; ++s) {
        const cd a = y[s], b = w[(size_t)e * wstep];
        re += a.real() * b.real() - a.imag() * b.imag();
        im += a.real() * b.imag() + a.imag() * b.real();
        e += x;
        if (e >= len) e -= len;
      }
      out[x] = cd(re, im);
    }
  }
}

// separable inverse DFT with the 1/n already folded into the input: out[x] = sum_k in[k] e^{+2 pi i k.x/m}
void idft_separable(int dim, int m, std::vector<cd>& a) {
  std::vector<cd> tw(m);
  for (int j = 0; j < m; ++j) tw[j] = cd(std::cos(2.0 * kPi * j / m), std::sin(2.0 * kPi * j / m));
  std::vector<cd> line(m), res(m);
  const int n = (dim == 3) ? m * m * m : m * m;
  for (int axis = 0; axis < dim; ++axis) {
    const int stride = axis == 0 ? 1 : (axis == 1 ? m : m * m);
    for (int outer = 0; outer < n / (m * stride); ++outer)
      for (int inner = 0; inner < stride; ++inner) {
        const size_t base = (size_t)outer * m * stride + inner;
        for (int t = 0; t < m; ++t) line[t] = a[base + (size_t)t * stride];
        dft_plus(line.data(), 1, res.data(), m, tw.data(), 1, m);
        for (int t = 0; t < m; ++t) a[base + (size_t)t * stride] = res[t];
      }
  }
}

// R factor (cols x cols, column-major, upper triangular) of the Householder QR of B (rows x
// cols, column-major, overwritten by the reflectors): B = Q R, so R has the singular values
// and right singular vectors of B, and the Jacobi sweeps run on cols x cols.
void householder_r(std::vector<cd>& B, int rows, int cols, std::vector<cd>& R) {
  R.assign((size_t)cols * cols, cd(0.0, 0.0));
  for (int k = 0; k < cols; ++k) {
    cd* bk = &B[(size_t)k * rows];
    double tail = 0.0;
    for (int i = k + 1; i < rows; ++i) tail += std::norm(bk[i]);
    const cd x0 = bk[k];
    const double ax0 = std::abs(x0), xn = std::sqrt(ax0 * ax0 + tail);
    cd alpha(0.0, 0.0);
    if (xn > 0.0) {
      // v = x - alpha e_k with alpha = -e^{i arg x0} |x|: |v|^2 = (|x0| + |x|)^2 + tail, no cancellation
      const cd ph = ax0 > 0.0 ? x0 / ax0 : cd(1.0, 0.0);
      alpha = -ph * xn;
      bk[k] = x0 - alpha;
      const double vn2 = (ax0 + xn) * (ax0 + xn) + tail;
      for (int j = k + 1; j < cols; ++j) {
        cd* bj = &B[(size_t)j * rows];
        cd w(0.0, 0.0);
        for (int i = k; i < rows; ++i) w += std::conj(bk[i]) * bj[i];
        const cd f = 2.0 * w / vn2;
        for (int i = k; i < rows; ++i) bj[i] -= f * bk[i];
      }
    }
    R[(size_t)k * cols + k] = alpha;
    for (int j = k + 1; j < cols; ++j) R[(size_t)j * cols + k] = B[(size_t)j * rows + k];
  }
}

// one-sided Jacobi on the columns of B (rows x cols, column-major); returns V (cols x
// cols, column-major) with B V having orthogonal columns.
void one_sided_jacobi(std::vector<cd>& B, int rows, int cols, std::vector<cd>& V) {
  V.assign((size_t)cols * cols, cd(0.0, 0.0));
  for (int i = 0; i < cols; ++i) V[(size_t)i * cols + i] = 1.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    bool rotated = false;
    for (int p = 0; p < cols - 1; ++p)
      for (int q = p + 1; q < cols; ++q) {
        cd* bp = &B[(size_t)p * rows];
        cd* bq = &B[(size_t)q * rows];
        double al = 0.0, be = 0.0;
        cd ga(0.0, 0.0);
        for (int i = 0; i < rows; ++i) {
          al += std::norm(bp[i]);
          be += std::norm(bq[i]);
          ga += std::conj(bp[i]) * bq[i];
        }
        const double ag = std::abs(ga);
        if (ag <= 1e-15 * std::sqrt(al * be) || ag == 0.0) continue;
        rotated = true;
        const cd eth = ga / ag;                 // e^{i theta}
        const double zeta = (be - al) / (2.0 * ag);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        // b_p' = c b_p - s e^{-i th} b_q ; b_q' = s e^{i th} b_p + c b_q
        const cd sm = s * std::conj(eth), sp = s * eth;
        for (int i = 0; i < rows; ++i) {
          const cd x = bp[i], y = bq[i];
          bp[i] = c * x - sm * y;
          bq[i] = sp * x + c * y;
        }
        cd* vp = &V[(size_t)p * cols];
        cd* vq = &V[(size_t)q * cols];
        for (int i = 0; i < cols; ++i) {
          const cd x = vp[i], y = vq[i];
          vp[i] = c * x - sm * y;
          vq[i] = sp * x + c * y;
        }
      }
    if (!rotated) break;
  }
}

// y[0..len) -= a x[0..len) on the interleaved (re, im) doubles of std::complex arrays: a
// plain loop that compilers vectorise (std::complex products keep a scalar inf/nan path)
inline void caxpy_sub(int len, cd a, const cd* x, cd* y) {
  const double ar = a.real(), ai = a.imag();
  const double* xd = reinterpret_cast<const double*>(x);
  double* yd = reinterpret_cast<double*>(y);
  for (int j = 0; j < len; ++j) {
    const double xr = xd[2 * j], xi = xd[2 * j + 1];
    yd[2 * j] -= ar * xr - ai * xi;
    yd[2 * j + 1] -= ar * xi + ai * xr;
  }
}

// Partial LU without pivoting of the first ns rows / columns of the nf x nf row-major
// front F: on return F holds the unit-lower multipliers, U, and in its trailing
// (nf - ns)^2 block the Schur complement.  Blocked right-looking elimination: inside a
// panel of kPanel pivots each pivot row is first brought fully up to date (its part
// beyond the panel receives the panel's earlier pivots), so every pivot sees its whole
// updated row exactly as in unblocked elimination; then the rows below the panel get the
// panel's rank-kPanel update one row at a time, with the panel's rows of U in cache.
// Rows and terms with a zero multiplier are skipped.  A pivot below pivot_floor times the
// largest entry of its updated row is raised to that size (static pivoting) and counted.
// Pivot statistics of the static pivoting, accumulated per thread and merged
struct PivotStats {
  double pmin = 1e300, pmax = 0.0;
  int nperturbed = 0;
};

void partial_lu(cd* F, int nf, int ns, double pivot_floor, PivotStats& out) {
  constexpr int kPanel = 32;
  const cd zero(0.0, 0.0);
  for (int kb = 0; kb < ns; kb += kPanel) {
    const int ke = std::min(kb + kPanel, ns);
    for (int k = kb; k < ke; ++k) {
      cd* rk = F + (size_t)k * nf;
      for (int p = kb; p < k; ++p)
        if (rk[p] != zero) caxpy_sub(nf - ke, rk[p], F + (size_t)p * nf + ke, rk + ke);
      cd piv = rk[k];
      double rown = 0.0;
      for (int j = k; j < nf; ++j) rown = std::max(rown, std::abs(rk[j]));
      const double ap = std::abs(piv);
      if (ap < pivot_floor * rown || ap == 0.0) {
        const double mag = pivot_floor * (rown > 0.0 ? rown : 1.0);
        piv = (ap > 0.0) ? piv / ap * mag : cd(mag, 0.0);
        rk[k] = piv;
        ++out.nperturbed;
      }
      out.pmin = std::min(out.pmin, std::abs(piv));
      out.pmax = std::max(out.pmax, std::abs(piv));
      const cd ip = 1.0 / piv;
      for (int i = k + 1; i < nf; ++i) {
        cd* ri = F + (size_t)i * nf;
        if (ri[k] == zero) continue;
        const cd l = ri[k] * ip;
        ri[k] = l;
        caxpy_sub(ke - k - 1, l, rk + k + 1, ri + k + 1);   // the panel's columns only
      }
    }
    for (int i = ke; i < nf; ++i) {                          // F22 -= L21 U12
      cd* ri = F + (size_t)i * nf;
      for (int p = kb; p < ke; ++p)
        if (ri[p] != zero) caxpy_sub(nf - ke, ri[p], F + (size_t)p * nf + ke, ri + ke);
    }
  }
}

}  // namespace

SppStructure spp_build_structure(int dim, int m, int r) {
  SppStructure st;
  st.dim = dim;
  st.m = m;
  st.r = r;
  st.n = (dim == 3) ? m * m * m : m * m;
  Builder bd{dim, m, r, &st, {}, {}, {}, {}};
  Box top;
  for (int d = 0; d < 3; ++d) {
    top.lo[d] = 0;
    top.ext[d] = d < dim ? m : 1;
    top.per[d] = d < dim;
  }
  bd.nd(top);
  const int nn = (int)bd.node_pts.size();
  // ND numbering
  st.perm.clear();
  st.iperm.assign(st.n, -1);
  st.nodes.resize(nn);
  for (int i = 0; i < nn; ++i) {
    st.nodes[i].off = (int)st.perm.size();
    st.nodes[i].ns = (int)bd.node_pts[i].size();
    st.nodes[i].parent = -1;
    for (int p : bd.node_pts[i]) {
      st.iperm[p] = (int)st.perm.size();
      st.perm.push_back(p);
    }
  }
  for (int i = 0; i < nn; ++i) {
    if (bd.node_children_a[i] >= 0) st.nodes[bd.node_children_a[i]].parent = i;
    if (bd.node_children_b[i] >= 0) st.nodes[bd.node_children_b[i]].parent = i;
  }
  // heights (postorder: children first)
  for (int i = 0; i < nn; ++i) {
    int h = 0;
    if (bd.node_children_a[i] >= 0) h = std::max(h, st.nodes[bd.node_children_a[i]].height + 1);
    if (bd.node_children_b[i] >= 0) h = std::max(h, st.nodes[bd.node_children_b[i]].height + 1);
    st.nodes[i].height = h;
  }
  // boundaries
  long long fo = 0;
  int uo = 0;
  for (int i = 0; i < nn; ++i) {
    std::vector<int> hal;
    bd.halo(bd.node_box[i], hal);
    std::vector<std::pair<int, int>> b;
    for (int p : hal) b.push_back({st.iperm[p], p});
    std::sort(b.begin(), b.end());
    SppNode& nd = st.nodes[i];
    nd.nb = (int)b.size();
    nd.boff = (int)st.bnd.size();
    for (auto& e : b) {
      st.bnd.push_back(e.first);
      st.bnat.push_back(e.second);
    }
    nd.uoff = uo;
    uo += nd.nb;
    nd.wf = fo;
    nd.wb = fo + (long long)(nd.ns + nd.nb) * nd.ns;
    fo = nd.wb + (long long)nd.ns * (nd.ns + nd.nb);
    st.max_ns = std::max(st.max_ns, nd.ns);
    st.max_nb = std::max(st.max_nb, nd.nb);
  }
  st.urows = uo;
  st.factor_size = fo;
  // levels
  int H = 0;
  for (auto& nd : st.nodes) H = std::max(H, nd.height);
  st.levels.assign(H + 1, {});
  for (int i = 0; i < nn; ++i) st.levels[st.nodes[i].height].push_back(i);
  for (int hgt = 0; hgt <= H; ++hgt) {
    st.fstart.push_back((int)st.fblocks.size() / 2);
    st.bstart.push_back((int)st.bblocks.size() / 2);
    for (int id : st.levels[hgt]) {
      const SppNode& nd = st.nodes[id];
      for (int r0 = 0; r0 < nd.ns + nd.nb; r0 += SppStructure::RB) { st.fblocks.push_back(id); st.fblocks.push_back(r0); }
      for (int r0 = 0; r0 < nd.ns; r0 += SppStructure::RB) { st.bblocks.push_back(id); st.bblocks.push_back(r0); }
    }
    st.fcount.push_back((int)st.fblocks.size() / 2 - st.fstart.back());
    st.bcount.push_back((int)st.bblocks.size() / 2 - st.bstart.back());
    int fk = 0, bk = 0;
    for (int id : st.levels[hgt]) {
      fk = std::max(fk, st.nodes[id].ns);
      bk = std::max(bk, st.nodes[id].ns + st.nodes[id].nb);
    }
    st.fkmax.push_back(fk);
    st.bkmax.push_back(bk);
  }
  // contributions: row r receives u[uoff_D + pos] for every node D with bnd_D[pos] = r
  std::vector<std::vector<int>> rows(st.n);
  for (int i = 0; i < nn; ++i) {
    const SppNode& nd = st.nodes[i];
    for (int pos = 0; pos < nd.nb; ++pos) rows[st.bnd[nd.boff + pos]].push_back(nd.uoff + pos);
  }
  st.contrib_ptr.assign(st.n + 1, 0);
  for (int rr = 0; rr < st.n; ++rr) st.contrib_ptr[rr + 1] = st.contrib_ptr[rr] + (int)rows[rr].size();
  st.contrib_idx.reserve(st.contrib_ptr[st.n]);
  for (int rr = 0; rr < st.n; ++rr) st.contrib_idx.insert(st.contrib_idx.end(), rows[rr].begin(), rows[rr].end());
  // leaf data: bandwidth from the stencil couplings inside each leaf, halo couplings.
  // 2D only: a cell of a 2D box couples to at most NBR = 3^2 halo cells; 3D leaves (up to
  // 19 halo couplings per cell) keep their dense W blocks and run with the other levels.
  if (dim == 2) {
    std::vector<int> ischild(nn, 0);
    for (int i = 0; i < nn; ++i) {
      if (bd.node_children_a[i] >= 0) ischild[i] = 1;
      if (bd.node_children_b[i] >= 0) ischild[i] = 1;
    }
    // periodic Chebyshev distance between grid points, from their coordinates
    std::vector<int> crd((size_t)st.n * 2);
    for (int p = 0; p < st.n; ++p) {
      crd[2 * (size_t)p] = p % m;
      crd[2 * (size_t)p + 1] = p / m;
    }
    auto cheb = [&](int p, int q) {
      int tx = std::abs(crd[2 * (size_t)p] - crd[2 * (size_t)q]);
      int ty = std::abs(crd[2 * (size_t)p + 1] - crd[2 * (size_t)q + 1]);
      tx = std::min(tx, m - tx);
      ty = std::min(ty, m - ty);
      return std::max(tx, ty);
    };
    long long vo = 0;
    for (int i = 0; i < nn; ++i) {
      if (bd.node_children_a[i] >= 0 || bd.node_children_b[i] >= 0) continue;
      const SppNode& nd = st.nodes[i];
      int bw = 0;
      for (int a = 0; a < nd.ns; ++a)
        for (int b2 = 0; b2 < nd.ns; ++b2)
          if (cheb(st.perm[nd.off + a], st.perm[nd.off + b2]) <= r) bw = std::max(bw, std::abs(a - b2));
      st.leaf_bw = std::max(st.leaf_bw, bw);
    }
    for (int i = 0; i < nn; ++i) {
      if (bd.node_children_a[i] >= 0 || bd.node_children_b[i] >= 0) continue;
      const SppNode& nd = st.nodes[i];
      st.leaf_nodes.push_back(i);
      st.leaf_voff.push_back(vo);
      vo += (long long)nd.ns * st.leaf_bw + (long long)nd.ns * (st.leaf_bw + 1) + (long long)nd.nb * SppStructure::NBR +
            (long long)nd.ns * SppStructure::NBR;
      st.leaf_ioff_bs.push_back((int)st.leaf_bs_idx.size());
      for (int j = 0; j < nd.nb; ++j) {
        int t = 0;
        for (int a = 0; a < nd.ns && t < SppStructure::NBR; ++a)
          if (cheb(st.bnat[nd.boff + j], st.perm[nd.off + a]) <= r) { st.leaf_bs_idx.push_back(a); ++t; }
        for (; t < SppStructure::NBR; ++t) st.leaf_bs_idx.push_back(-1);
      }
      st.leaf_ioff_sb.push_back((int)st.leaf_sb_idx.size());
      for (int a = 0; a < nd.ns; ++a) {
        int t = 0;
        for (int j = 0; j < nd.nb && t < SppStructure::NBR; ++j)
          if (cheb(st.perm[nd.off + a], st.bnat[nd.boff + j]) <= r) { st.leaf_sb_idx.push_back(j); ++t; }
        for (; t < SppStructure::NBR; ++t) st.leaf_sb_idx.push_back(-1);
      }
    }
    st.leaf_size = vo;
  }
  // stencil offsets, x fastest
  const int rz = dim == 3 ? r : 0;
  for (int dz = -rz; dz <= rz; ++dz)
    for (int dy = -r; dy <= r; ++dy)
      for (int dx = -r; dx <= r; ++dx) {
        st.offsets.push_back(dx);
        st.offsets.push_back(dy);
        st.offsets.push_back(dz);
      }
  return st;
}

void green_symbol(int dim, int m, double kin, double lmean, double shift, cd z, std::vector<cd>& ghat) {
  const int n = (dim == 3) ? m * m * m : m * m;
  ghat.resize(n);
  auto sk = [m](int i) { return i < (m + 1) / 2 ? i : i - m; };   // DFT order; the same as m / 2 for even m
  for (int i = 0; i < n; ++i) {
    const int ix = i % m, iy = (i / m) % m, iz = (dim == 3) ? i / (m * m) : 0;
    const double k2 = (double)sk(ix) * sk(ix) + (double)sk(iy) * sk(iy) + (dim == 3 ? (double)sk(iz) * sk(iz) : 0.0);
    ghat[i] = 1.0 / (kin * k2 + lmean - shift - z) / (double)n;
  }
}

void spp_pole_stencil(const SppStructure& st, double kin, const double* V, double shift, cd z, SppStencil& out,
                      std::vector<cd>& ghat) {
  const int dim = st.dim, m = st.m, n = st.n;
  double lmean = 0.0;
  for (int i = 0; i < n; ++i) lmean += V[i];
  lmean /= n;
  out.lmean = lmean;
  green_symbol(dim, m, kin, lmean, shift, z, ghat);
  std::vector<cd> g(ghat);
  idft_separable(dim, m, g);   // g[x] = G(x, 0)
  const int na = (int)st.offsets.size() / 3;
  auto off_flat = [&](int dx, int dy, int dz) {
    return wrap(dx, m) + m * (wrap(dy, m) + (dim == 3 ? m * wrap(dz, m) : 0));
  };
  auto coord = [&](int p, int& x, int& y, int& zc) {
    x = p % m;
    y = (p / m) % m;
    zc = dim == 3 ? p / (m * m) : 0;
  };
  std::vector<int> a0(na);
  for (int i = 0; i < na; ++i) a0[i] = off_flat(st.offsets[3 * i], st.offsets[3 * i + 1], st.offsets[3 * i + 2]);
  std::vector<char> in_a(n, 0);
  for (int p : a0) in_a[p] = 1;
  const int rows = n - na;
  // B = G(a, a^c)^*: column i holds conj(G(o_i, c)) = conj(g[o_i - c]) over c not in a
  std::vector<cd> B((size_t)na * rows);
  for (int i = 0; i < na; ++i) {
    const int ox = st.offsets[3 * i], oy = st.offsets[3 * i + 1], oz = st.offsets[3 * i + 2];
    int row = 0;
    for (int c = 0; c < n; ++c) {
      if (in_a[c]) continue;
      int cx, cy, cz;
      coord(c, cx, cy, cz);
      B[(size_t)i * rows + row] = std::conj(g[off_flat(ox - cx, oy - cy, oz - cz)]);
      ++row;
    }
  }
  std::vector<cd> R, Vj;
  householder_r(B, rows, na, R);
  one_sided_jacobi(R, na, na, Vj);
  int jmin = 0;
  double smin = 1e300, smax = 0.0;
  for (int j = 0; j < na; ++j) {
    double s = 0.0;
    for (int i = 0; i < na; ++i) s += std::norm(R[(size_t)j * na + i]);
    s = std::sqrt(s);
    if (s < smin) { smin = s; jmin = j; }
    smax = std::max(smax, s);
  }
  out.sigma_min = smin;
  out.sigma_max = smax;
  out.q.resize(na);
  for (int i = 0; i < na; ++i) out.q[i] = std::conj(Vj[(size_t)jmin * na + i]);
  // (qG)(0, a_j) = sum_i q_i G(o_i, o_j) = sum_i q_i g[o_i - o_j]
  out.qg.assign(na, cd(0.0, 0.0));
  for (int j = 0; j < na; ++j)
    for (int i = 0; i < na; ++i)
      out.qg[j] += out.q[i] * g[off_flat(st.offsets[3 * i] - st.offsets[3 * j],
                                         st.offsets[3 * i + 1] - st.offsets[3 * j + 1],
                                         st.offsets[3 * i + 2] - st.offsets[3 * j + 2])];
}

void spp_setup_pole(const SppStructure& st, double kin, const double* V, double shift, cd z, double pivot_floor,
                    SppPole& out, std::vector<cd>& ghat, int threads) {
  const int dim = st.dim, m = st.m, n = st.n;
  SppStencil sten;
  spp_pole_stencil(st, kin, V, shift, z, sten, ghat);
  out.q = sten.q;
  out.sigma_min = sten.sigma_min;
  out.sigma_max = sten.sigma_max;
  const std::vector<cd>& qg = sten.qg;
  const double lmean = sten.lmean;
  const int na = (int)st.offsets.size() / 3;
  auto off_flat = [&](int dx, int dy, int dz) {
    return wrap(dx, m) + m * (wrap(dy, m) + (dim == 3 ? m * wrap(dz, m) : 0));
  };
  auto coord = [&](int p, int& x, int& y, int& zc) {
    x = p % m;
    y = (p / m) % m;
    zc = dim == 3 ? p / (m * m) : 0;
  };
  // P(row j, stencil t) = q_t + qg_t (V_{j+o_t} - l)
  auto neighbor = [&](int p, int t) {
    int x, y, zc;
    coord(p, x, y, zc);
    return off_flat(x + st.offsets[3 * t], y + st.offsets[3 * t + 1], zc + st.offsets[3 * t + 2]);
  };
  auto pval = [&](int row, int t) { return out.q[t] + qg[t] * (V[neighbor(row, t)] - lmean); };
  // ---- multifrontal LU
  out.factor.assign((size_t)st.factor_size, cd(0.0, 0.0));
  out.leafval.assign((size_t)st.leaf_size, cd(0.0, 0.0));
  const int nn = (int)st.nodes.size();
  std::vector<std::vector<cd>> upd(nn);
  std::vector<std::vector<int>> children(nn);
  for (int i = 0; i < nn; ++i)
    if (st.nodes[i].parent >= 0) children[st.nodes[i].parent].push_back(i);
  // One supernode: assemble its front from P's couplings and its children's update
  // matrices (in the fixed order of `children`), eliminate, store W_f / W_b (and the
  // banded leaf data), keep the update matrix for the parent.  It reads only its own
  // front, its children's update matrices and st, and writes only its own slices of
  // out.factor / out.leafval and upd[s]: nodes whose subtrees are disjoint can run on
  // different threads, each with its own loc (unknown -> front position) and stats.
  auto factor_node = [&](int s, std::vector<int>& loc, PivotStats& ps) {
    const SppNode& nd = st.nodes[s];
    const int ns = nd.ns, nb = nd.nb, nf = ns + nb;
    for (int i = 0; i < ns; ++i) loc[nd.off + i] = i;
    for (int j = 0; j < nb; ++j) loc[st.bnd[nd.boff + j]] = ns + j;
    std::vector<cd> F((size_t)nf * nf, cd(0.0, 0.0));
    for (int i = 0; i < ns; ++i) {
      const int nat = st.perm[nd.off + i];
      for (int t = 0; t < na; ++t) {
        // row entry P(nat, nat + o_t)
        const int jn = st.iperm[neighbor(nat, t)];
        if (loc[jn] >= 0) F[(size_t)i * nf + loc[jn]] += pval(nat, t);
        // column entry P(rnat, nat) where rnat + o_t = nat
        int x, y, zc;
        coord(nat, x, y, zc);
        const int rnat = off_flat(x - st.offsets[3 * t], y - st.offsets[3 * t + 1], zc - st.offsets[3 * t + 2]);
        const int jr = st.iperm[rnat];
        if (loc[jr] >= ns) F[(size_t)loc[jr] * nf + i] += pval(rnat, t);
      }
    }
    for (int c : children[s]) {
      const SppNode& cn = st.nodes[c];
      const std::vector<cd>& U = upd[c];
      for (int a = 0; a < cn.nb; ++a) {
        const int la = loc[st.bnd[cn.boff + a]];
        for (int b = 0; b < cn.nb; ++b) F[(size_t)la * nf + loc[st.bnd[cn.boff + b]]] += U[(size_t)a * cn.nb + b];
      }
      std::vector<cd>().swap(upd[c]);
    }
    const bool leaf = children[s].empty() && !st.leaf_nodes.empty();   // banded leaf data (2D) is kept
    std::vector<cd> F0;
    if (leaf) F0 = F;   // original couplings of the leaf (no children: F holds only P's entries)
    partial_lu(F.data(), nf, ns, pivot_floor, ps);
    // W_f = [L_SS^-1 ; L_BS L_SS^-1], W_b = [U_SS^-1 , -U_SS^-1 U_SB]: with these, each
    // supernode's forward and backward step is one dense product on the device.  All four
    // are formed row by row from contiguous rows (zero coefficients skipped).
    const cd zero(0.0, 0.0);
    std::vector<cd> Li((size_t)ns * ns, zero), Ui((size_t)ns * ns, zero);
    for (int i = 0; i < ns; ++i) {           // L Li = I: Li(i,:) = e_i - sum_{k<i} L(i,k) Li(k,:)
      cd* li = &Li[(size_t)i * ns];
      li[i] = 1.0;
      const cd* lrow = &F[(size_t)i * nf];
      for (int k = 0; k < i; ++k)
        if (lrow[k] != zero) caxpy_sub(k + 1, lrow[k], &Li[(size_t)k * ns], li);
    }
    for (int i = ns - 1; i >= 0; --i) {      // U Ui = I: Ui(i,:) = (e_i - sum_{k>i} U(i,k) Ui(k,:)) / U(i,i)
      cd* ui = &Ui[(size_t)i * ns];
      ui[i] = 1.0;
      const cd* urow = &F[(size_t)i * nf];
      for (int k = i + 1; k < ns; ++k)
        if (urow[k] != zero) caxpy_sub(ns - k, urow[k], &Ui[(size_t)k * ns + k], ui + k);
      const cd d = 1.0 / urow[i];
      for (int j = i; j < ns; ++j) ui[j] *= d;
    }
    cd* wf = &out.factor[nd.wf];
    cd* wb = &out.factor[nd.wb];
    std::copy(Li.begin(), Li.end(), wf);
    for (int i = 0; i < nb; ++i) {           // L_BS Li
      cd* w = wf + (size_t)(ns + i) * ns;
      std::fill(w, w + ns, zero);
      const cd* lrow = &F[(size_t)(ns + i) * nf];
      for (int k = 0; k < ns; ++k)
        if (lrow[k] != zero) caxpy_sub(k + 1, -lrow[k], &Li[(size_t)k * ns], w);
    }
    const int kb = ns + nb;
    for (int i = 0; i < ns; ++i) {           // [Ui , -Ui U_SB]
      cd* w = wb + (size_t)i * kb;
      std::copy(&Ui[(size_t)i * ns], &Ui[(size_t)i * ns] + ns, w);
      std::fill(w + ns, w + kb, zero);
      for (int k = i; k < ns; ++k)
        if (w[k] != zero) caxpy_sub(nb, w[k], &F[(size_t)k * nf + ns], w + ns);
    }
    if (leaf) {
      const int bw = st.leaf_bw, NB = SppStructure::NBR;
      const size_t li = std::lower_bound(st.leaf_nodes.begin(), st.leaf_nodes.end(), s) - st.leaf_nodes.begin();
      cd* v = &out.leafval[st.leaf_voff[li]];
      cd* Lb = v;
      cd* Ub = Lb + (size_t)ns * bw;
      cd* Fbs = Ub + (size_t)ns * (bw + 1);
      cd* Fsb = Fbs + (size_t)nb * NB;
      for (int i = 0; i < ns; ++i) {
        for (int t = 0; t < bw; ++t) {
          const int j = i - 1 - t;
          Lb[(size_t)i * bw + t] = j >= 0 ? F[(size_t)i * nf + j] : cd(0.0, 0.0);
        }
        for (int t = 0; t <= bw; ++t) {
          const int j = i + t;
          Ub[(size_t)i * (bw + 1) + t] = j < ns ? (t == 0 ? 1.0 / F[(size_t)i * nf + i] : F[(size_t)i * nf + j]) : cd(0.0, 0.0);
        }
      }
      const int* bsi = &st.leaf_bs_idx[st.leaf_ioff_bs[li]];
      for (int j = 0; j < nb; ++j)
        for (int t = 0; t < NB; ++t) {
          const int i = bsi[j * NB + t];
          Fbs[(size_t)j * NB + t] = i >= 0 ? F0[(size_t)(ns + j) * nf + i] : cd(0.0, 0.0);
        }
      const int* sbi = &st.leaf_sb_idx[st.leaf_ioff_sb[li]];
      for (int i = 0; i < ns; ++i)
        for (int t = 0; t < NB; ++t) {
          const int j = sbi[i * NB + t];
          Fsb[(size_t)i * NB + t] = j >= 0 ? F0[(size_t)i * nf + ns + j] : cd(0.0, 0.0);
        }
    }
    upd[s].resize((size_t)nb * nb);
    for (int i = 0; i < nb; ++i)
      for (int j = 0; j < nb; ++j) upd[s][(size_t)i * nb + j] = F[(size_t)(ns + i) * nf + ns + j];
    for (int i = 0; i < ns; ++i) loc[nd.off + i] = -1;
    for (int j = 0; j < nb; ++j) loc[st.bnd[nd.boff + j]] = -1;
  };
  // Tree schedule: a node is ready once its children are factorised; with one thread this
  // is the index (post-) order.  Every node's arithmetic is the same on any thread, so the
  // factor is bitwise independent of the thread count.
  const int T = std::max(1, std::min(threads, 16));
  std::vector<PivotStats> stats(T);
  if (T == 1) {
    std::vector<int> loc(n, -1);
    for (int s = 0; s < nn; ++s) factor_node(s, loc, stats[0]);
  } else {
    std::vector<int> pending(nn), ready;
    for (int s = 0; s < nn; ++s) {
      pending[s] = (int)children[s].size();
      if (pending[s] == 0) ready.push_back(s);
    }
    std::mutex mu;
    std::condition_variable cv;
    int done = 0;
    auto worker = [&](int t) {
      std::vector<int> loc(n, -1);
      std::unique_lock<std::mutex> lk(mu);
      for (;;) {
        cv.wait(lk, [&] { return !ready.empty() || done == nn; });
        if (ready.empty()) return;                 // every node is factorised
        const int s = ready.back();                // depth first: the most recently readied node
        ready.pop_back();
        lk.unlock();
        factor_node(s, loc, stats[t]);
        lk.lock();
        ++done;
        const int par = st.nodes[s].parent;
        if (par >= 0 && --pending[par] == 0) ready.push_back(par);
        cv.notify_all();
      }
    };
    std::vector<std::thread> pool;
    for (int t = 1; t < T; ++t) pool.emplace_back(worker, t);
    worker(0);
    for (auto& th : pool) th.join();
  }
  out.pivot_min = 1e300;
  out.pivot_max = 0.0;
  out.nperturbed = 0;
  for (const PivotStats& ps : stats) {
    out.pivot_min = std::min(out.pivot_min, ps.pmin);
    out.pivot_max = std::max(out.pivot_max, ps.pmax);
    out.nperturbed += ps.nperturbed;
  }
}

SppFactorMaps spp_factor_maps(const SppStructure& st) {
  SppFactorMaps mp;
  const int dim = st.dim, m = st.m, n = st.n;
  const int na = (int)st.offsets.size() / 3;
  const int nn = (int)st.nodes.size();
  auto off_flat = [&](int dx, int dy, int dz) {
    return wrap(dx, m) + m * (wrap(dy, m) + (dim == 3 ? m * wrap(dz, m) : 0));
  };
  auto coord = [&](int p, int& x, int& y, int& zc) {
    x = p % m;
    y = (p / m) % m;
    zc = dim == 3 ? p / (m * m) : 0;
  };
  mp.nbr.resize((size_t)n * na);
  for (int p = 0; p < n; ++p) {
    int x, y, zc;
    coord(p, x, y, zc);
    for (int t = 0; t < na; ++t)
      mp.nbr[(size_t)p * na + t] =
          off_flat(x + st.offsets[3 * t], y + st.offsets[3 * t + 1], zc + st.offsets[3 * t + 2]);
  }
  mp.foff.resize(nn);
  mp.child0.assign(nn, -1);
  mp.child1.assign(nn, -1);
  mp.leaf_of.assign(nn, -1);
  for (int i = 0; i < nn; ++i) {
    mp.foff[i] = mp.front_size;
    const long long nf = st.nodes[i].ns + st.nodes[i].nb;
    mp.front_size += nf * nf;
    const int par = st.nodes[i].parent;
    if (par >= 0) {
      if (mp.child0[par] < 0) mp.child0[par] = i;
      else if (mp.child1[par] < 0) mp.child1[par] = i;
      else return mp;   // more than two children: not a bisection tree
    }
  }
  for (size_t li = 0; li < st.leaf_nodes.size(); ++li) mp.leaf_of[st.leaf_nodes[li]] = (int)li;
  // P's entries of each front (the row and column couplings of its own unknowns, as the
  // host factorisation assembles them), and the place of each boundary unknown in the
  // parent's front
  std::vector<int> loc(n, -1);
  mp.emap.assign(st.bnd.size(), -1);
  mp.asm_ptr.assign(nn + 1, 0);
  std::vector<int> seen;
  for (int s = 0; s < nn; ++s) {
    const SppNode& nd = st.nodes[s];
    const int ns = nd.ns, nb = nd.nb, nf = ns + nb;
    for (int i = 0; i < ns; ++i) loc[nd.off + i] = i;
    for (int j = 0; j < nb; ++j) loc[st.bnd[nd.boff + j]] = ns + j;
    const size_t first = mp.asm_pos.size();
    for (int i = 0; i < ns; ++i) {
      const int nat = st.perm[nd.off + i];
      int x, y, zc;
      coord(nat, x, y, zc);
      for (int t = 0; t < na; ++t) {
        const int jn = st.iperm[mp.nbr[(size_t)nat * na + t]];
        if (loc[jn] >= 0) {
          mp.asm_pos.push_back(i * nf + loc[jn]);
          mp.asm_src.push_back(nat * na + t);
        }
        const int rnat = off_flat(x - st.offsets[3 * t], y - st.offsets[3 * t + 1], zc - st.offsets[3 * t + 2]);
        const int jr = st.iperm[rnat];
        if (loc[jr] >= ns) {
          mp.asm_pos.push_back(loc[jr] * nf + i);
          mp.asm_src.push_back(rnat * na + t);
        }
      }
    }
    seen.assign(mp.asm_pos.begin() + first, mp.asm_pos.end());
    std::sort(seen.begin(), seen.end());
    if (std::adjacent_find(seen.begin(), seen.end()) != seen.end()) return mp;   // two entries on one position
    mp.asm_ptr[s + 1] = (int)mp.asm_pos.size();
    for (int c : {mp.child0[s], mp.child1[s]}) {
      if (c < 0) continue;
      const SppNode& cn = st.nodes[c];
      for (int a = 0; a < cn.nb; ++a) mp.emap[cn.boff + a] = loc[st.bnd[cn.boff + a]];
    }
    for (int i = 0; i < ns; ++i) loc[nd.off + i] = -1;
    for (int j = 0; j < nb; ++j) loc[st.bnd[nd.boff + j]] = -1;
  }
  for (int s = 0; s < nn; ++s)
    if (st.nodes[s].parent >= 0)
      for (int a = 0; a < st.nodes[s].nb; ++a)
        if (mp.emap[st.nodes[s].boff + a] < 0) return mp;   // a boundary unknown missing from the parent's front
  mp.ok = true;
  return mp;
}

}  // namespace omm
