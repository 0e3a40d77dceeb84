// C ABI of the OMM library: handle, device memory, pole setup and the iteration driver.
//
// One preconditioned CG step (Algorithm 1) on the device, with H = H0 - sigma and the
// unshifted H0 X kept (the shift enters only the FP64 N x N algebra):
//   Grad = 2 H0X - X (K0 + 2 sigma (I - S)) - H0X S          (Sec. 2.1, rearranged)
//   G = -sum_j w_j Y_j, (H - z_j) Y_j = Grad by batched GMRES  (Sec. 3.1 eqs. direct, lst)
//   beta = Re<G, G - G_prev> / <G_prev, G_prev>, D = G + beta D (Polak-Ribiere)
//   HD = H0 D; Grams [X D]^*[X D H0X H0D]; quartic c_0..c_4; exact line search t
//   X += t D, H0X += t H0D; the Grams of the new X follow from the quartic expansion.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "factor.h"
#include "kernels.h"
#include "spp.h"
#include "trsv.h"

using namespace omm;

namespace {

thread_local std::string g_last_error;
void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_free)(void*, void*) = nullptr;
void* g_alloc_ctx = nullptr;
std::mutex g_alloc_mu;

constexpr int PMAX = 32;
constexpr int KMAXB = 16;

}  // namespace

void omm_internal_set_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  g_last_error = std::string(cudaGetErrorString(e)) + " in " + what + " (" + file + ":" + std::to_string(line) + ")";
}

static void omm_internal_set_message(const char* msg) { g_last_error = msg; }

enum ProfClass { PC_HAPPLY = 0, PC_GREENQ, PC_TRSV, PC_ORTH, PC_GRAM, PC_BLOCKUPD, PC_VEC, PC_SMALL, PC_TRSV_LEAF, PC_NCLS };
const char* const kProfNames[PC_NCLS] = {"happly", "greenq", "trsv_levels", "orth", "gram", "block_update", "vector",
                                         "small", "trsv_leaf"};

struct Prof {
  bool on = false;
  double ms[PC_NCLS] = {};
  long long calls[PC_NCLS] = {};
  long long kernels[PC_NCLS] = {};
  double bytes[PC_NCLS] = {};        // algorithmic bytes (what the step must move)
  double impl_bytes[PC_NCLS] = {};   // this implementation's own byte model (intermediates included)
  double flops[PC_NCLS] = {};        // algorithmic real flops (classes whose bound is arithmetic)
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<std::pair<int, size_t>> pending;   // class, first event index
};

struct omm_ctx {
  int dim = 2, m = 0;
  size_t n = 0;
  int N = 0;
  double L = 1.0, shift = 0.0, kin = 0.0, lmean = 0.0;
  omm_params prm{};
  bool dbl = true;
  size_t csz = 16;
  cudaStream_t st = nullptr;
  // extra streams for the triangular solves of groups of poles (forked from and joined to st)
  static constexpr int kTrsvStreams = 8;
  cudaStream_t st2[kTrsvStreams] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kTrsvStreams] = {};
  void* (*alloc)(size_t, void*) = nullptr;
  void (*release)(void*, void*) = nullptr;
  void* alloc_ctx = nullptr;
  std::vector<void*> allocs;
  size_t bytes = 0;
  std::vector<double> Vh;

  // device state
  void* V = nullptr;       // n reals (working precision)
  void* V64 = nullptr;     // n doubles (FP64 check)
  void* tw = nullptr;      // m twiddles (working precision)
  void* tw64 = nullptr;
  void* blk = nullptr;     // [X | D | HX | HD], each N columns
  void* Grad = nullptr;
  void* G = nullptr;
  void* Gp = nullptr;
  double2* gram = nullptr;  // 2N x 4N
  void* gram_work = nullptr;
  void* sc_block = nullptr;     // OmmScalars, then the line search's scratch
  double* ls_work = nullptr;    // N x 12 doubles: partial traces of the line search
  void* M1 = nullptr;
  void* M2 = nullptr;
  OmmScalars* sc = nullptr;
  OmmScalars* sc_h = nullptr;  // pinned
  void* red_work = nullptr;
  double2* shifts = nullptr;   // [PMAX] sigma + z_p
  double2* zero_shift = nullptr;
  double2* tmp_shift = nullptr;
  double2* wts = nullptr;      // [PMAX] w_p
  int* nact_d = nullptr;
  int* nact_h = nullptr;       // pinned
  // FP64 check work
  void* X64 = nullptr;
  void* HX64 = nullptr;
  double2* gram64 = nullptr;
  void* gram64_work = nullptr;
  void* fft_tmp = nullptr;
  size_t fft_tmp_bytes = 0;
  void* tc_work = nullptr;      // tensor-core Gram split-K partials
  size_t tc_work_bytes = 0;
  int* tc_err = nullptr;        // set by the tensor-core Gram if a bounded wait gave up
  void* gw_dbg = nullptr;       // Gram work for omm_gram / the residual check
  size_t gw_dbg_bytes = 0;
  void* m64 = nullptr;          // residual-check N x N matrices and two norms
  int Pfac = 0;                 // poles the factor buffers are sized for
  // allocation groups: set only once every buffer of the group exists and is initialised,
  // so that a failed allocation is retried in full by the next call (a byte or pole count
  // is likewise reset before its buffer is replaced)
  bool fp64_ready = false, ghat_ready = false, proj_ready = false;
  bool breakdown = false;       // the last CG run met a non-finite energy / step / beta
  bool enqueue_only = false;    // omm_solve_enqueue: no host synchronisation, results stay on the device
  double2* sigma64 = nullptr;   // (sigma, 0) on the device for the FP64 check
  bool enqueued = false;        // results of an omm_solve_enqueue are waiting on the device

  // poles
  int P = 0;
  std::vector<double2> z, w;   // the poles solved (conjugate pairs folded for real orbitals)
  bool real_combine = false;   // pole sum keeps 2 Re(w Y) of each folded pair
  // precomputed preconditioner U U^* (Algorithm 2)
  bool use_proj = false;
  void* Uproj = nullptr;        // n x N, orthonormal columns
  void* projM = nullptr;        // N x N working-precision coefficient block
  void* projZero = nullptr;     // N x N zeros (second operand of the block update)
  double2* projC = nullptr;     // up to 2N x 2N FP64 Gram
  void* projY64 = nullptr;      // 3 x n x N complex128: [Y1 | Y2] being orthonormalised and a product
  void* projM64 = nullptr;      // 2N x N complex128 coefficient block
  void* projZero64 = nullptr;   // N x N complex128 zeros
  void* projWork64 = nullptr;   // FP64 Gram work
  bool poles_set = false;
  // Fourier-diagonal comparison preconditioner (gTPA, Sec. 2.2)
  bool use_gtpa = false;
  void* gtpa_tab = nullptr;     // 2 x n working precision: +g_t(s_k)/n, then -g_t(s_k)/n
  void* gtpa_one = nullptr;     // the one-point stencil {1} of the Green kernel
  // GMRES work (sized for P poles)
  int Palloc = 0;
  void* Vb = nullptr;
  void* Zb = nullptr;
  void* xs = nullptr;
  void* wv = nullptr;
  void* tv = nullptr;
  double2* Hh = nullptr;
  double2* cs = nullptr;
  double2* gv = nullptr;
  double2* yv = nullptr;
  double* beta = nullptr;
  double* bnorm = nullptr;
  int* active = nullptr;
  int* steps = nullptr;
  int* itot = nullptr;
  double* est = nullptr;
  // inner preconditioner data
  void* ghat = nullptr;   // P * n (working precision)
  void* qd = nullptr;     // P * nq
  int nq = 1;
  // sparsifying factor
  SppStructure spp;
  bool spp_built = false;
  std::vector<SppPole> spp_poles;
  void* factor = nullptr;
  void* ynd = nullptr;
  void* xnd = nullptr;    // assembled right-hand sides, then solutions, ND order (S x n)
  void* ubuf = nullptr;
  int* d_node_ns = nullptr;
  int* d_node_nb = nullptr;
  int* d_node_off = nullptr;
  int* d_node_boff = nullptr;
  int* d_node_uoff = nullptr;
  long long* d_node_wf = nullptr;
  long long* d_node_wb = nullptr;
  int* d_perm = nullptr;
  int* d_bnat = nullptr;
  int* d_bnd = nullptr;
  int* d_iperm = nullptr;       // natural -> ND index (the Green kernel's store order)
  int* d_cptr = nullptr;
  int* d_cidx = nullptr;
  int* d_fblocks = nullptr;
  int* d_leaf_nodes = nullptr;
  long long* d_leaf_voff = nullptr;
  int* d_leaf_ioff_bs = nullptr;
  int* d_leaf_ioff_sb = nullptr;
  int* d_leaf_bs_idx = nullptr;
  int* d_leaf_sb_idx = nullptr;
  void* leafvals = nullptr;     // P * leaf_size complex
  int* d_bblocks = nullptr;
  int* d_lunk = nullptr;                    // unknowns of each tree height (ND indices)
  unsigned* d_trsv_bar = nullptr;           // grid barrier of the persistent level launch: count, generation, error
  // device factorisation of P (k_factor.cu): maps built once per handle
  bool fmaps_tried = false, fmaps_ok = false;
  long long front_size = 0;                 // front entries per pole
  long long* d_foff = nullptr;
  int *d_child0 = nullptr, *d_child1 = nullptr, *d_asm_ptr = nullptr, *d_asm_pos = nullptr, *d_asm_src = nullptr;
  int *d_nbr = nullptr, *d_emap = nullptr, *d_leaf_of = nullptr, *d_hnodes = nullptr;
  double* d_Vdbl = nullptr;
  double2* d_qq = nullptr;                  // PMAX x 27 (q) then PMAX x 27 ((qG)(0, a))
  std::vector<FactorHeight> fheights;       // per height: launch shapes (node ids in d_hnodes)
  bool last_factor_device = false;
  // algorithmic complex elements of the triangular-solve phases: per system and per pole
  double tb_leaf_fwd_sys = 0, tb_leaf_bwd_sys = 0, tb_leaf_pole = 0, tb_lvl_sys = 0, tb_lvl_pole = 0;
  double n_leaf = 0, n_sep = 0;   // unknowns in the leaves / in the separators (algorithmic bytes)
  long long nact_last = -1;   // systems active after the last count (-1: unknown); algorithmic bytes
                              // of masked launches count these only
  std::vector<int> lunk_start, lunk_count;
  size_t trsv_smem = 0;
  double cur_rtol = 0.0;       // GMRES tolerance of the current round (gmres_rtol, then refilter_rtol)
  int last_gmres_max = 0;
  double last_relres_max = 0.0;
  int gmres_total = 0;

  Prof prof;

  void prof_flush() {
    if (prof.pending.empty()) return;
    cudaStreamSynchronize(st);
    for (auto& pe : prof.pending) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, prof.pool[pe.second], prof.pool[pe.second + 1]) == cudaSuccess) prof.ms[pe.first] += t;
    }
    prof.pending.clear();
    prof.used = 0;
  }
  size_t prof_event_pair() {
    if (prof.used + 2 > prof.pool.size()) {
      if (prof.pool.size() < 4096) {
        while (prof.pool.size() < 4096) {
          cudaEvent_t e;
          if (cudaEventCreate(&e) != cudaSuccess) break;
          prof.pool.push_back(e);
        }
      }
      if (prof.used + 2 > prof.pool.size()) prof_flush();
    }
    const size_t i = prof.used;
    prof.used += 2;
    return i;
  }

  ~omm_ctx() {
    prof.pending.clear();
    for (cudaEvent_t e : prof.pool) cudaEventDestroy(e);
    if (ev_fork) cudaEventDestroy(ev_fork);
    for (int i = 0; i < kTrsvStreams; ++i) {
      if (ev_join[i]) cudaEventDestroy(ev_join[i]);
      if (st2[i]) cudaStreamDestroy(st2[i]);
    }
    for (void* p : allocs) {
      if (release) release(p, alloc_ctx);
      else cudaFree(p);
    }
    if (sc_h) cudaFreeHost(sc_h);
    if (nact_h) cudaFreeHost(nact_h);
  }

  // a work buffer that does not outlive the call: freed again by dfree (same size)
  void dfree(void* p, size_t b) {
    auto it = std::find(allocs.begin(), allocs.end(), p);
    if (!p || it == allocs.end()) return;
    allocs.erase(it);
    if (release) release(p, alloc_ctx);
    else cudaFree(p);
    if (b == 0) b = 16;
    bytes -= (b + 255) / 256 * 256;
  }
  omm_status dalloc(void** p, size_t b) {
    *p = nullptr;
    if (b == 0) b = 16;
    b = (b + 255) / 256 * 256;
    if (alloc) {
      *p = alloc(b, alloc_ctx);
      if (!*p) return OMM_ENOMEM;
    } else {
      cudaError_t e = cudaMalloc(p, b);
      if (e != cudaSuccess) {
        omm_internal_set_cuda_error(e, "cudaMalloc", __FILE__, __LINE__);
        *p = nullptr;
        return OMM_ENOMEM;
      }
    }
    allocs.push_back(*p);
    bytes += b;
    return OMM_OK;
  }
  template <typename P_>
  omm_status dalloc_t(P_** p, size_t b) {
    void* v = nullptr;
    omm_status s = dalloc(&v, b);
    *p = (P_*)v;
    return s;
  }
  void* col(void* base, size_t j) const { return (char*)base + j * n * csz; }
  void* X() const { return col(blk, 0); }
  void* D() const { return col(blk, N); }
  void* HX() const { return col(blk, 2 * N); }
  void* HD() const { return col(blk, 3 * N); }
};

namespace {

omm_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return OMM_OK;
  omm_internal_set_cuda_error(e, what, __FILE__, __LINE__);
  return OMM_ECUDA;
}

// Times one launch group on the handle's stream when profiling is on; always counts the
// kernels launched and their algorithmic bytes.
struct ProfScope {
  omm_ctx* h;
  int cls;
  size_t ev = (size_t)-1;
  ProfScope(omm_ctx* h_, int cls_, double bytes, int nk, double impl = -1.0) : h(h_), cls(cls_) {
    h->prof.calls[cls] += 1;
    h->prof.kernels[cls] += nk;
    h->prof.bytes[cls] += bytes;
    h->prof.impl_bytes[cls] += impl >= 0.0 ? impl : bytes;
    if (h->prof.on) {
      ev = h->prof_event_pair();
      cudaEventRecord(h->prof.pool[ev], h->st);
    }
  }
  ~ProfScope() {
    if (ev != (size_t)-1) {
      cudaEventRecord(h->prof.pool[ev + 1], h->st);
      h->prof.pending.push_back({cls, ev});
    }
  }
};
#define PROF(cls, bytes, nk, expr)                 \
  do {                                             \
    ProfScope _ps(h, (cls), (double)(bytes), (nk)); \
    OMM_TRY(expr);                                 \
  } while (0)
// the same with the implementation's own byte count beside the algorithmic one
#define PROF2(cls, bytes, impl, nk, expr)                            \
  do {                                                               \
    ProfScope _ps(h, (cls), (double)(bytes), (nk), (double)(impl)); \
    OMM_TRY(expr);                                                   \
  } while (0)

double kinetic_max(int dim, int m, double L) {
  const double c = 2.0 * M_PI * M_PI / (L * L);
  return c * dim * (double)(m / 2) * (m / 2);
}

bool radix_ok(int m) {
  if (m < 2) return false;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  return m == 1;
}

omm_status ensure_fft_tmp(omm_ctx* h, size_t ncols, bool dbl);

// columns a masked launch touches (for its algorithmic bytes): the active count when known
double live_cols(const omm_ctx* h, double ncols, const int* active) {
  return (active && h->nact_last >= 0) ? std::min(ncols, (double)h->nact_last) : ncols;
}

// H0 X (shift 0) or (H0 - s_g) X for ncols columns; fused single-CTA kernel when the grid
// fits shared memory, else the multi-pass kernels
omm_status happly(omm_ctx* h, const void* X, void* Y, int ncols, const double2* shifts, int cpg, const int* active,
                  bool fp64 = false) {
  const bool dbl = fp64 || h->dbl;
  const void* V = fp64 ? h->V64 : h->V;
  const void* tw = fp64 ? h->tw64 : h->tw;
  const double kn = h->kin / (double)h->n;
  const double bytes = (2.0 * live_cols(h, ncols, active) * (dbl ? 16 : 8) + (dbl ? 8 : 4)) * (double)h->n;
  if (fused_fft_supported(h->dim, h->m, dbl)) {
    PROF(PC_HAPPLY, bytes, 1,
         cuda_status(launch_happly(dbl, h->dim, h->m, X, Y, ncols, V, shifts, cpg, tw, kn, active, h->st), "happly"));
    return OMM_OK;
  }
  OMM_TRY(ensure_fft_tmp(h, ncols, dbl));
  PROF(PC_HAPPLY, bytes, big_fft_launches(h->dim, h->m, dbl, false),
       cuda_status(launch_happly_big(dbl, h->dim, h->m, X, Y, ncols, V, shifts, cpg, tw, kn, active, h->fft_tmp, h->st),
                   "happly"));
  return OMM_OK;
}

omm_status greenq(omm_ctx* h, const void* B, void* Out, int ncols, int nq, int cpg, const int* active,
                  const void* ghat = nullptr, const void* q = nullptr, const int* iperm = nullptr) {
  if (!ghat) ghat = h->ghat;
  if (!q) q = h->qd;
  const double bytes = (2.0 * live_cols(h, ncols, active) + (double)((ncols + cpg - 1) / cpg)) * h->csz * (double)h->n;
  if (fused_fft_supported(h->dim, h->m, h->dbl)) {
    PROF(PC_GREENQ, bytes, 1,
         cuda_status(launch_greenq(h->dbl, h->dim, h->m, B, Out, ncols, ghat, q, nq, cpg, h->tw, active, iperm, h->st),
                     "greenq"));
    return OMM_OK;
  }
  OMM_TRY(ensure_fft_tmp(h, ncols, h->dbl));
  PROF(PC_GREENQ, bytes, big_fft_launches(h->dim, h->m, h->dbl, true),
       cuda_status(
           launch_greenq_big(h->dbl, h->dim, h->m, B, Out, ncols, ghat, q, nq, cpg, h->tw, active, iperm, h->fft_tmp,
                             h->st),
           "greenq"));
  return OMM_OK;
}

omm_status ensure_dbg_work(omm_ctx* h, size_t need) {
  if (h->gw_dbg_bytes >= need) return OMM_OK;
  h->gw_dbg_bytes = 0;
  OMM_TRY(h->dalloc(&h->gw_dbg, need));
  h->gw_dbg_bytes = need;
  return OMM_OK;
}

omm_status ensure_fft_tmp(omm_ctx* h, size_t ncols, bool dbl) {
  const size_t need = ncols * h->n * (dbl ? 16 : 8);
  if (h->fft_tmp_bytes >= need) return OMM_OK;
  h->fft_tmp_bytes = 0;
  OMM_TRY(h->dalloc(&h->fft_tmp, need));   // the old buffer stays owned until destroy
  h->fft_tmp_bytes = need;
  return OMM_OK;
}

omm_status upload_twiddles(omm_ctx* h, void* dst, bool dbl) {
  std::vector<double> t(2 * h->m);
  for (int k = 0; k < h->m; ++k) {
    t[2 * k] = std::cos(2.0 * M_PI * k / h->m);
    t[2 * k + 1] = -std::sin(2.0 * M_PI * k / h->m);
  }
  if (dbl) return cuda_status(cudaMemcpyAsync(dst, t.data(), t.size() * 8, cudaMemcpyHostToDevice, h->st), "tw");
  std::vector<float> f(t.begin(), t.end());
  omm_status s = cuda_status(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->st), "tw");
  if (s == OMM_OK) s = cuda_status(cudaStreamSynchronize(h->st), "tw sync");
  return s;
}

omm_status upload_complex(omm_ctx* h, void* dst, const std::vector<cd>& v, bool dbl) {
  if (dbl)
    return cuda_status(cudaMemcpyAsync(dst, v.data(), v.size() * 16, cudaMemcpyHostToDevice, h->st), "upload");
  std::vector<float> f(2 * v.size());
  for (size_t i = 0; i < v.size(); ++i) {
    f[2 * i] = (float)v[i].real();
    f[2 * i + 1] = (float)v[i].imag();
  }
  omm_status s = cuda_status(cudaMemcpyAsync(dst, f.data(), f.size() * 4, cudaMemcpyHostToDevice, h->st), "upload");
  if (s == OMM_OK) s = cuda_status(cudaStreamSynchronize(h->st), "upload sync");
  return s;
}

template <typename T_>
omm_status upload_vec(omm_ctx* h, T_** dst, const std::vector<T_>& v) {
  OMM_TRY(h->dalloc_t(dst, v.size() * sizeof(T_)));
  if (v.empty()) return OMM_OK;
  return cuda_status(cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T_), cudaMemcpyHostToDevice, h->st), "upload");
}

omm_status ensure_gmres_work(omm_ctx* h, int P) {
  if (h->Palloc >= P) return OMM_OK;
  h->Palloc = 0;
  const size_t S = (size_t)P * h->N;
  const size_t vb = S * h->n * h->csz;
  const int m = h->prm.gmres_m;
  OMM_TRY(h->dalloc(&h->Vb, vb * (m + 1)));
  OMM_TRY(h->dalloc(&h->Zb, vb * m));
  OMM_TRY(h->dalloc(&h->xs, vb));
  OMM_TRY(h->dalloc(&h->wv, vb));
  OMM_TRY(h->dalloc(&h->tv, vb));
  OMM_TRY(h->dalloc_t(&h->Hh, S * (KMAXB + 1) * KMAXB * sizeof(double2)));
  OMM_TRY(h->dalloc_t(&h->cs, S * KMAXB * 2 * sizeof(double2)));
  OMM_TRY(h->dalloc_t(&h->gv, S * (KMAXB + 1) * sizeof(double2)));
  OMM_TRY(h->dalloc_t(&h->yv, S * KMAXB * sizeof(double2)));
  OMM_TRY(h->dalloc_t(&h->beta, S * sizeof(double)));
  OMM_TRY(h->dalloc_t(&h->bnorm, S * sizeof(double)));
  OMM_TRY(h->dalloc_t(&h->active, S * sizeof(int)));
  OMM_TRY(h->dalloc_t(&h->steps, S * sizeof(int)));
  OMM_TRY(h->dalloc_t(&h->itot, S * sizeof(int)));
  OMM_TRY(h->dalloc_t(&h->est, S * sizeof(double)));
  h->Palloc = P;
  return OMM_OK;
}

TrsvArgs trsv_args(omm_ctx* h, int Ncols, size_t S) {
  TrsvArgs a;
  a.node_ns = h->d_node_ns;
  a.node_nb = h->d_node_nb;
  a.node_off = h->d_node_off;
  a.node_boff = h->d_node_boff;
  a.node_uoff = h->d_node_uoff;
  a.node_wf = h->d_node_wf;
  a.node_wb = h->d_node_wb;
  a.perm = h->d_perm;
  a.bnat = h->d_bnat;
  a.bnd = h->d_bnd;
  a.contrib_ptr = h->d_cptr;
  a.contrib_idx = h->d_cidx;
  a.factor_size = h->spp.factor_size;
  a.n = h->n;
  a.N = Ncols;
  a.S = S;
  return a;
}

LeafArgs leaf_args(omm_ctx* h, int pole_base) {
  LeafArgs la;
  const SppStructure& s = h->spp;
  la.nleaves = (int)s.leaf_nodes.size();
  la.bw = s.leaf_bw;
  for (int id : s.leaf_nodes) {
    la.max_ns = std::max(la.max_ns, s.nodes[id].ns);
    la.max_nb = std::max(la.max_nb, s.nodes[id].nb);
  }
  la.nodes = h->d_leaf_nodes;
  la.voff = h->d_leaf_voff;
  la.ioff_bs = h->d_leaf_ioff_bs;
  la.ioff_sb = h->d_leaf_ioff_sb;
  la.bs_idx = h->d_leaf_bs_idx;
  la.sb_idx = h->d_leaf_sb_idx;
  la.leaf_size = s.leaf_size;
  la.vals = (const char*)h->leafvals + (size_t)pole_base * s.leaf_size * h->csz;
  return la;
}

TrsvLevels trsv_levels(omm_ctx* h) {
  TrsvLevels lv;
  lv.nlevels = (int)h->spp.levels.size();
  lv.fblocks = h->d_fblocks;
  lv.bblocks = h->d_bblocks;
  lv.fstart = h->spp.fstart;
  lv.fcount = h->spp.fcount;
  lv.bstart = h->spp.bstart;
  lv.bcount = h->spp.bcount;
  lv.fkmax = h->spp.fkmax;
  lv.bkmax = h->spp.bkmax;
  lv.lunk = h->d_lunk;
  lv.ustart = h->lunk_start;
  lv.ucount = h->lunk_count;
  return lv;
}

// Right preconditioner for S = P*N systems: Z = M^-1 V (natural order in and out)
omm_status inner_apply(omm_ctx* h, int P, int Ncols, const void* Vk, void* Z, const int* active, void* tmp) {
  const int inner = h->prm.inner;
  const size_t S = (size_t)P * Ncols;
  if (inner == OMM_INNER_NONE) {
    return cuda_status(cudaMemcpyAsync(Z, Vk, S * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "copy");
  }
  if (inner == OMM_INNER_KINETIC) return greenq(h, Vk, Z, (int)S, 1, Ncols, active);
  // Green kernel + Q stencil, stored in the nested-dissection order of the solves
  OMM_TRY(greenq(h, Vk, tmp, (int)S, h->nq, Ncols, active, nullptr, nullptr, h->d_iperm));
  TrsvArgs a = trsv_args(h, Ncols, S);
  TrsvLevels lv = trsv_levels(h);
  const LeafArgs la = leaf_args(h, 0);
  const bool has_leaves = la.nleaves > 0;
  const double cs = (double)h->csz;
  const double Se = live_cols(h, (double)S, active);
  int nk = 0;
  for (int l = has_leaves ? 1 : 0; l < lv.nlevels; ++l)   // per height: (assembly +) product forward, product backward
    nk += (lv.fcount[l] > 0) * (1 + (lv.ucount[l] > 0)) + (lv.bcount[l] > 0);
  // Groups of poles on their own streams: the latency-bound top of the tree of one group
  // overlaps the other groups' work.  Every per-pole array is offset on the host; the update
  // rows keep their row stride S and are offset by columns.
  const int ng = std::min(P, h->prm.trsv_streams > 0 ? h->prm.trsv_streams : (int)omm_ctx::kTrsvStreams);
  if (ng > 1 && !h->st2[0]) {
    OMM_TRY(cuda_status(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming), "event"));
    for (int g = 0; g < omm_ctx::kTrsvStreams; ++g) {
      OMM_TRY(cuda_status(cudaStreamCreateWithFlags(&h->st2[g], cudaStreamNonBlocking), "stream"));
      OMM_TRY(cuda_status(cudaEventCreateWithFlags(&h->ev_join[g], cudaEventDisableTiming), "event"));
    }
  }
  auto spp = [&](int phases) -> omm_status {
    if (phases == (SPP_LEVELS_FWD | SPP_LEVELS_BWD) && h->prm.trsv_persistent) {
      // every height of every pole in one cooperative launch (falls back to the launches per
      // height below when the structure does not fit it)
      bool done = false;
      OMM_TRY(cuda_status(launch_spp_levels_persistent(h->dbl, a, lv, has_leaves, P, tmp, h->ynd, h->ubuf, Z, h->xnd,
                                                       h->factor, active, h->d_trsv_bar, h->st, &done),
                          "spp levels"));
      if (done) return OMM_OK;
    }
    if (ng == 1 || (h->prm.trsv_persistent && phases != (SPP_LEVELS_FWD | SPP_LEVELS_BWD)))
      return cuda_status(launch_spp_solve(phases, h->dbl, a, lv, la, P, tmp, h->ynd, h->ubuf, Z, h->xnd, h->factor,
                                          active, h->trsv_smem, h->prm.launch_overlap, h->st),
                         "spp");
    OMM_TRY(cuda_status(cudaEventRecord(h->ev_fork, h->st), "fork"));
    int p0 = 0;
    for (int g = 0; g < ng; ++g) {
      const int pg = P / ng + (g < P % ng ? 1 : 0);   // poles of group g
      const size_t sys0 = (size_t)p0 * Ncols;
      const size_t vec0 = sys0 * h->n * h->csz;
      OMM_TRY(cuda_status(cudaStreamWaitEvent(h->st2[g], h->ev_fork, 0), "fork"));
      OMM_TRY(cuda_status(
          launch_spp_solve(phases, h->dbl, a, lv, leaf_args(h, p0), pg, (const char*)tmp + vec0,
                           (char*)h->ynd + vec0, (char*)h->ubuf + sys0 * h->csz, (char*)Z + vec0,
                           (char*)h->xnd + vec0,
                           (const char*)h->factor + (size_t)p0 * h->spp.factor_size * h->csz,
                           active ? active + sys0 : nullptr, h->trsv_smem, h->prm.launch_overlap, h->st2[g]),
          "spp"));
      OMM_TRY(cuda_status(cudaEventRecord(h->ev_join[g], h->st2[g]), "join"));
      OMM_TRY(cuda_status(cudaStreamWaitEvent(h->st, h->ev_join[g], 0), "join"));
      p0 += pg;
    }
    return OMM_OK;
  };
  const int ns = h->prm.trsv_persistent ? 1 : ng;   // launches per kernel (one per stream)
  if (h->prm.trsv_persistent) nk = 1;   // (the fallback per height counts as one too)
  // Algorithmic bytes of the triangular solves (L then U): each unknown's right-hand side
  // read and y written, y read and x written (4 per unknown and active system), and each
  // pole's factor read once (leaf values split over the two leaf passes).  The
  // implementation's own model adds the update rows, the assembled separator right-hand
  // sides and the boundary gathers.
  if (has_leaves)
    PROF2(PC_TRSV_LEAF, (2.0 * h->n_leaf * Se + 0.5 * h->tb_leaf_pole * P) * cs,
          (h->tb_leaf_fwd_sys * Se + h->tb_leaf_pole * P) * cs, ns, spp(SPP_LEAF_FWD));
  // the supernode products: every W_f and W_b entry of a pole times each of its active
  // systems, 8 real flops per complex multiply-add
  h->prof.flops[PC_TRSV] += 8.0 * h->tb_lvl_pole * Se;
  PROF2(PC_TRSV, (4.0 * h->n_sep * Se + h->tb_lvl_pole * P) * cs, (h->tb_lvl_sys * Se + h->tb_lvl_pole * P) * cs,
        ns * nk, spp(SPP_LEVELS_FWD | SPP_LEVELS_BWD));
  if (has_leaves)
    PROF2(PC_TRSV_LEAF, (2.0 * h->n_leaf * Se + 0.5 * h->tb_leaf_pole * P) * cs,
          (h->tb_leaf_bwd_sys * Se + h->tb_leaf_pole * P) * cs, ns, spp(SPP_LEAF_BWD));
  return OMM_OK;
}

omm_status read_nactive(omm_ctx* h, int* out) {
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->nact_h, h->nact_d, sizeof(int), cudaMemcpyDeviceToHost, h->st), "nact"));
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "nact sync"));
  *out = *h->nact_h;
  h->nact_last = *out;
  return OMM_OK;
}

// out = sign * sum_p w_p Y_p, (H - sigma - z_p) Y_p = R by GMRES from Y_p = R
omm_status pole_solve(omm_ctx* h, const void* R, void* out, double sign) {
  const int P = h->P, N = h->N;
  KrylovDims d;
  d.S = P * N;
  d.N = N;
  d.n = h->n;
  d.m = h->prm.gmres_m;
  const size_t vs = (size_t)d.S * h->n * h->csz;
  auto Vk = [&](int k) { return (void*)((char*)h->Vb + (size_t)k * vs); };
  auto Zk = [&](int k) { return (void*)((char*)h->Zb + (size_t)k * vs); };
  const double rtol = h->cur_rtol;
  const int fixed = h->prm.gmres_fixed;
  // the host reads the active counts to stop early, except when the solve is only being
  // enqueued: then every cycle runs all its steps, and systems that met the tolerance are
  // masked on the device (their kernels return at once)
  const bool host_checks = !fixed && !h->enqueue_only;
  OMM_TRY(cuda_status(cudaMemsetAsync(h->itot, 0, sizeof(int) * d.S, h->st), "memset"));
  for (int cyc = 0; cyc < h->prm.gmres_cycles; ++cyc) {
    h->nact_last = -1;   // every system until the cycle start has been counted
    OMM_TRY(cuda_status(cudaMemsetAsync(h->steps, 0, sizeof(int) * d.S, h->st), "memset"));
    if (cyc == 0) {
      OMM_TRY(happly(h, R, h->wv, N, h->zero_shift, N, nullptr));
      PROF(PC_VEC, 3.0 * d.S * h->n * h->csz, 1,
           cuda_status(launch_krylov_init0(h->dbl, d, R, h->wv, h->shifts, Vk(0), h->xs, h->beta, h->gv, h->bnorm,
                                           h->active, rtol, fixed, h->st),
                       "init0"));
    } else {
      OMM_TRY(happly(h, h->xs, h->wv, d.S, h->shifts, N, nullptr));
      PROF(PC_VEC, 3.0 * d.S * h->n * h->csz, 1,
           cuda_status(launch_krylov_restart(h->dbl, d, R, h->wv, Vk(0), h->beta, h->gv, h->bnorm, h->active, rtol,
                                             fixed, h->st),
                       "restart"));
    }
    double cyc_cols = d.S;   // systems the cycle works on (for the update's bytes)
    if (host_checks) {
      // count active systems after the cycle start
      PROF(PC_SMALL, 0, 1, cuda_status(launch_count_active(d, h->active, h->nact_d, h->st), "count"));
      int na = 0;
      OMM_TRY(read_nactive(h, &na));
      if (na == 0) break;
      cyc_cols = na;
    }
    int steps_run = 0;
    for (int k = 0; k < d.m; ++k) {
      ++steps_run;
      OMM_TRY(inner_apply(h, P, N, Vk(k), Zk(k), h->active, h->tv));
      OMM_TRY(happly(h, Zk(k), h->wv, d.S, h->shifts, N, h->active));
      // algorithmic: the k + 1 basis vectors and w read once, V_{k+1} written; the kernels
      // stream the basis and w once per sweep, three times
      PROF2(PC_ORTH, (k + 3.0) * live_cols(h, d.S, h->active) * h->n * h->csz,
            (3.0 * k + 7.0) * live_cols(h, d.S, h->active) * h->n * h->csz, 1,
            cuda_status(launch_krylov_orth(h->dbl, d, k, h->Vb, h->wv, h->Hh, h->active, h->st), "orth"));
      OMM_TRY(cuda_status(cudaMemsetAsync(h->nact_d, 0, sizeof(int), h->st), "memset"));
      PROF(PC_SMALL, 0, 1,
           cuda_status(launch_krylov_givens(d, k, h->Hh, h->cs, h->gv, h->bnorm, h->active, h->steps, h->est, rtol,
                                            fixed, h->nact_d, h->st),
                       "givens"));
      if (host_checks && k + 1 < d.m) {
        int na = 0;
        OMM_TRY(read_nactive(h, &na));
        if (na == 0) break;
      }
    }
    PROF(PC_VEC, (steps_run + 2.0) * cyc_cols * h->n * h->csz, 2,
         cuda_status(launch_krylov_update(h->dbl, d, h->Hh, h->gv, h->steps, h->yv, h->Zb, h->xs, h->itot, h->st),
                     "update"));
  }
  PROF(PC_VEC, (double)(d.S + N) * h->n * h->csz, 1,
       cuda_status(launch_pole_combine(h->dbl, d, P, h->wts, sign, h->real_combine, h->xs, out, h->st), "combine"));
  return OMM_OK;
}

omm_status gmres_stats(omm_ctx* h) {
  const int S = h->P * h->N;
  std::vector<int> it(S);
  std::vector<double> e(S);
  OMM_TRY(cuda_status(cudaMemcpyAsync(it.data(), h->itot, S * sizeof(int), cudaMemcpyDeviceToHost, h->st), "stats"));
  OMM_TRY(cuda_status(cudaMemcpyAsync(e.data(), h->est, S * sizeof(double), cudaMemcpyDeviceToHost, h->st), "stats"));
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "stats sync"));
  h->last_gmres_max = *std::max_element(it.begin(), it.end());
  h->last_relres_max = *std::max_element(e.begin(), e.end());
  return OMM_OK;
}

omm_status read_scalars(omm_ctx* h) {
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->sc_h, h->sc, sizeof(OmmScalars), cudaMemcpyDeviceToHost, h->st), "sc"));
  int e = 0;
  unsigned eb = 0;
  if (h->tc_err)
    OMM_TRY(cuda_status(cudaMemcpyAsync(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, h->st), "tc err"));
  if (h->d_trsv_bar)
    OMM_TRY(cuda_status(cudaMemcpyAsync(&eb, h->d_trsv_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, h->st),
                        "trsv err"));
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "sc sync"));
  if (eb) {
    // a bounded barrier wait of the persistent triangular solves gave up: clear the
    // barrier for the next launch and report it
    omm_internal_set_message("a grid barrier of the triangular solves timed out");
    OMM_TRY(cuda_status(cudaMemsetAsync(h->d_trsv_bar, 0, 4 * sizeof(unsigned), h->st), "memset"));
    return OMM_ETIMEOUT;
  }
  return e ? OMM_ETIMEOUT : OMM_OK;
}

// C = A^H B (complex double out): tensor cores for complex64 when enabled, else CUDA cores
omm_status gram_any(omm_ctx* h, const void* A, int na, const void* B, int nb, double2* C, int ldc, void* cc_work) {
  if (!h->dbl && h->prm.gram_tensor && gram_tc_supported(h->n)) {
    const size_t need = gram_tc_work_bytes(na, nb, h->n);
    if (need > h->tc_work_bytes) {
      h->tc_work_bytes = 0;
      OMM_TRY(h->dalloc(&h->tc_work, need));
      h->tc_work_bytes = need;
    }
    if (!h->tc_err) {
      int* flag = nullptr;
      OMM_TRY(h->dalloc_t(&flag, sizeof(int)));
      OMM_TRY(cuda_status(cudaMemsetAsync(flag, 0, sizeof(int), h->st), "memset"));
      h->tc_err = flag;
    }
    return cuda_status(launch_gram_tc(A, na, B, nb, h->n, C, ldc, h->tc_work, h->tc_err, h->st), "gram_tc");
  }
  return cuda_status(launch_gram(h->dbl, A, na, B, nb, h->n, C, ldc, cc_work, h->st), "gram");
}

// out = sign * U (U^* R): the precomputed preconditioner (one Gram, one block update)
omm_status apply_projector(omm_ctx* h, const void* R, void* out, double sign) {
  const int N = h->N;
  const double cnt = (double)N * h->n;
  PROF(PC_GRAM, 2.0 * cnt * h->csz, 2, gram_any(h, h->Uproj, N, R, N, h->projC, N, h->gram_work));
  PROF(PC_SMALL, 0, 1, cuda_status(launch_gram_to_matrix(h->dbl, h->projC, N, N, sign, h->projM, h->st), "projM"));
  PROF(PC_BLOCKUPD, 2.0 * cnt * h->csz, 1,
       cuda_status(launch_block_update(h->dbl, h->Uproj, h->Uproj, h->projM, h->projZero, 0.0, 0.0, N, h->n, out,
                                       h->st),
                   "proj"));
  return OMM_OK;
}

// out = sign * F^-1 (g_t(|k|^2 / tau) F R): one fused pass of the Green kernel with the
// gTPA table (1/n folded in) and the one-point stencil; real orbitals drop the rounding
// imaginary parts, as the pole sum does
omm_status apply_gtpa(omm_ctx* h, const void* R, void* out, double sign) {
  const void* tab = (const char*)h->gtpa_tab + (sign < 0 ? (size_t)h->n * h->csz : 0);
  OMM_TRY(greenq(h, R, out, h->N, 1, h->N, nullptr, tab, h->gtpa_one));
  if (h->prm.real_orbitals) {
    const size_t cnt = (size_t)h->N * h->n;
    PROF(PC_VEC, 1.0 * cnt * h->csz, 1, cuda_status(launch_real_part(h->dbl, cnt, out, h->st), "real"));
  }
  return OMM_OK;
}

// The preconditioner of the handle: gTPA while set, else U U^* once built, else the pole
// expansion
omm_status precondition(omm_ctx* h, const void* R, void* out, double sign) {
  if (h->use_gtpa) return apply_gtpa(h, R, out, sign);
  if (h->use_proj) return apply_projector(h, R, out, sign);
  return pole_solve(h, R, out, sign);
}

// Grams of the current X and the gradient update matrices (t = 0)
omm_status start_cg(omm_ctx* h) {
  OMM_TRY(happly(h, h->X(), h->HX(), h->N, h->zero_shift, h->N, nullptr));
  PROF(PC_GRAM, 5.0 * h->N * h->n * h->csz, 2,
       gram_any(h, h->X(), h->N, h->blk, 4 * h->N, h->gram, 4 * h->N, h->gram_work));
  PROF(PC_SMALL, 0, 1,
       cuda_status(launch_line_search(h->dbl, h->gram, h->N, h->shift, 0, h->prm.tol, h->sc, h->M1, h->M2, h->ls_work, h->st),
                   "ls0"));
  return OMM_OK;
}

omm_status cg_steps(omm_ctx* h, int k, omm_stats* st, int* done_iters, bool* conv) {
  h->breakdown = false;
  OMM_TRY(start_cg(h));
  const size_t cnt = (size_t)h->N * h->n;
  *conv = false;
  int it = 0;
  for (; it < k; ++it) {
    PROF(PC_BLOCKUPD, 3.0 * cnt * h->csz, 1,
         cuda_status(launch_block_update(h->dbl, h->X(), h->HX(), h->M1, h->M2, 0.0, 2.0, h->N, h->n, h->Grad, h->st),
                     "grad"));
    PROF(PC_VEC, 1.0 * cnt * h->csz, 2,
         cuda_status(launch_redot(h->dbl, cnt, h->Grad, h->Grad, &h->sc->grad2, h->red_work, h->st), "dot"));
    OMM_TRY(precondition(h, h->Grad, h->G, -1.0));
    PROF(PC_VEC, 2.0 * cnt * h->csz, 2,
         cuda_status(launch_redot(h->dbl, cnt, h->G, h->G, &h->sc->gg, h->red_work, h->st), "dot"));
    if (it > 0)
      PROF(PC_VEC, 2.0 * cnt * h->csz, 2,
           cuda_status(launch_redot(h->dbl, cnt, h->G, h->Gp, &h->sc->gdot, h->red_work, h->st), "dot"));
    PROF(PC_SMALL, 0, 1, cuda_status(launch_pr_beta(h->sc, it == 0 ? 1 : 0, h->st), "beta"));
    // D = G + beta D   (first step: D = G)
    if (it == 0)
      OMM_TRY(cuda_status(cudaMemcpyAsync(h->D(), h->G, cnt * h->csz, cudaMemcpyDeviceToDevice, h->st), "copy"));
    else
      PROF(PC_VEC, 3.0 * cnt * h->csz, 1,
           cuda_status(launch_axpby(h->dbl, cnt, nullptr, h->G, &h->sc->beta_c, h->D(), h->st), "dir"));
    OMM_TRY(happly(h, h->D(), h->HD(), h->N, h->zero_shift, h->N, nullptr));
    PROF(PC_GRAM, 6.0 * cnt * h->csz, 2, gram_any(h, h->blk, 2 * h->N, h->blk, 4 * h->N, h->gram, 4 * h->N, h->gram_work));
    PROF(PC_SMALL, 0, 1,
         cuda_status(launch_line_search(h->dbl, h->gram, h->N, h->shift, 1, h->prm.tol, h->sc, h->M1, h->M2, h->ls_work, h->st),
                     "ls"));
    // X += t D ; HX += t HD
    PROF(PC_VEC, 3.0 * cnt * h->csz, 1,
         cuda_status(launch_axpby(h->dbl, cnt, &h->sc->t_c, h->D(), &h->sc->one_c, h->X(), h->st), "upd"));
    PROF(PC_VEC, 3.0 * cnt * h->csz, 1,
         cuda_status(launch_axpby(h->dbl, cnt, &h->sc->t_c, h->HD(), &h->sc->one_c, h->HX(), h->st), "upd"));
    std::swap(h->G, h->Gp);
    if (h->enqueue_only) continue;   // fixed schedule: no host decision until the results are read
    OMM_TRY(read_scalars(h));
    if (!h->use_proj && !h->use_gtpa) {
      OMM_TRY(gmres_stats(h));
      h->gmres_total += h->last_gmres_max;
    }
    if (h->sc_h->bad) {
      *done_iters = it + 1;
      return OMM_ESHIFT;
    }
    if (!std::isfinite(h->sc_h->E1) || !std::isfinite(h->sc_h->t) || !std::isfinite(h->sc_h->beta)) {
      // numerical breakdown (a non-finite Gram, quartic or step): stop, not converged,
      // instead of iterating on NaN to maxit
      h->breakdown = true;
      omm_internal_set_message("non-finite energy, line-search step or beta in the CG");
      ++it;
      break;
    }
    if (h->sc_h->converged && !h->prm.fixed_iters) {
      *conv = true;
      ++it;
      break;
    }
  }
  if (h->prm.fixed_iters && it == k && !h->breakdown) *conv = true;   // the fixed schedule ran out
  *done_iters = it;
  if (st) {
    st->energy = h->sc_h->E1;
    st->grad_norm = std::sqrt(std::max(h->sc_h->grad2, 0.0));
    st->gmres_iters_max = h->last_gmres_max;
    st->gmres_relres_max = h->last_relres_max;
    st->gmres_iters_total = h->gmres_total;
  }
  return OMM_OK;
}


// FP64 check of the current X, all on the device: X converted to complex128, FP64 H-apply
// (shift sigma) and FP64 Gram C = X^*[X HX]; one CTA forms E_omm = tr K - 1/2 tr(S K)
// (eq. omm), the Cholesky factor S = R^* R and R^-1, two small products give -S^-1 K, and
// FP64 block updates form the Rayleigh-Ritz residual Res = HX - X S^-1 K (shift
// invariant) and the residual of the orthonormal basis Q = X R^-1 of span X,
// Res R^-1 = HQ - Q (Q^* H Q).  Outputs: *E; *resid = ||Res||_F / ||X||_F; *resid_orth =
// ||Res R^-1||_F (divided by the spectral gap it bounds the sine of the largest angle to
// the exact invariant subspace, Davis-Kahan).  A non-positive Cholesky pivot (X rank
// deficient) leaves both residuals NaN.
omm_status energy_fp64(omm_ctx* h, double* E, double* resid, double* resid_orth = nullptr) {
  const int N = h->N;
  const size_t cnt = (size_t)N * h->n;
  const size_t nn = (size_t)N * N;
  if (!h->fp64_ready) {
    OMM_TRY(h->dalloc(&h->X64, cnt * 16 * 4));   // [X | HX | Res | Res R^-1] in FP64
    OMM_TRY(h->dalloc_t(&h->gram64, (size_t)N * 2 * N * sizeof(double2)));
    OMM_TRY(h->dalloc(&h->gram64_work, gram_work_bytes(N, 2 * N, h->n)));
    OMM_TRY(h->dalloc_t(&h->tmp_shift, sizeof(double2) * 2));
    // N x N: R, R^-1, T, -S^-1 K, zeros; then E, three norms, the Cholesky flag
    OMM_TRY(h->dalloc(&h->m64, 5 * nn * 16 + 4 * sizeof(double) + sizeof(int)));
    OMM_TRY(cuda_status(cudaMemsetAsync((char*)h->m64 + 4 * nn * 16, 0, nn * 16, h->st), "memset"));
    OMM_TRY(h->dalloc_t(&h->sigma64, sizeof(double2)));
    const double2 sg = make_double2(h->shift, 0.0);
    OMM_TRY(cuda_status(cudaMemcpyAsync(h->sigma64, &sg, sizeof(sg), cudaMemcpyHostToDevice, h->st), "sigma"));
    OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "sync"));
    h->fp64_ready = true;
  }
  void* X64 = h->X64;
  void* HX64 = (char*)h->X64 + cnt * 16;
  void* R64 = (char*)h->X64 + 2 * cnt * 16;
  void* Q64 = (char*)h->X64 + 3 * cnt * 16;
  double2* Rc = (double2*)h->m64;
  double2* Rinv = Rc + nn;
  double2* T = Rc + 2 * nn;
  double2* Mneg = Rc + 3 * nn;
  const double2* Z0 = Rc + 4 * nn;
  double* dres = (double*)(Rc + 5 * nn);   // E, |Res|^2, |X|^2, |Res R^-1|^2
  int* dok = (int*)(dres + 4);
  if (h->dbl)
    OMM_TRY(cuda_status(cudaMemcpyAsync(X64, h->X(), cnt * 16, cudaMemcpyDeviceToDevice, h->st), "copy"));
  else
    PROF(PC_VEC, 24.0 * cnt, 1, cuda_status(launch_convert(true, cnt, h->X(), X64, h->st), "convert"));
  OMM_TRY(happly(h, X64, HX64, N, h->sigma64, N, nullptr, true));
  PROF(PC_GRAM, 3.0 * cnt * 16, 2,
       cuda_status(launch_gram(true, X64, N, X64, 2 * N, h->n, h->gram64, 2 * N, h->gram64_work, h->st), "gram64"));
  PROF(PC_SMALL, 0, 3,
       cuda_status(launch_fp64_check_small(h->gram64, 2 * N, N, dres, Rc, Rinv, T, Mneg, dok, h->st), "fp64 small"));
  if (resid) {
    PROF(PC_BLOCKUPD, 3.0 * cnt * 16, 1,
         cuda_status(launch_block_update(true, X64, HX64, Mneg, Z0, 0.0, 1.0, N, h->n, R64, h->st), "resid"));
    PROF(PC_BLOCKUPD, 2.0 * cnt * 16, 1,
         cuda_status(launch_block_update(true, R64, R64, Rinv, Z0, 0.0, 0.0, N, h->n, Q64, h->st), "resid orth"));
    PROF(PC_VEC, 2.0 * cnt * 16, 2, cuda_status(launch_redot(true, cnt, R64, R64, dres + 1, h->red_work, h->st), "dot"));
    PROF(PC_VEC, 2.0 * cnt * 16, 2, cuda_status(launch_redot(true, cnt, X64, X64, dres + 2, h->red_work, h->st), "dot"));
    PROF(PC_VEC, 2.0 * cnt * 16, 2, cuda_status(launch_redot(true, cnt, Q64, Q64, dres + 3, h->red_work, h->st), "dot"));
  }
  if (h->enqueue_only) return OMM_OK;   // read by omm_read_result
  double out[4] = {0.0, 0.0, 0.0, 0.0};
  int ok = 0;
  OMM_TRY(cuda_status(cudaMemcpyAsync(out, dres, sizeof(out), cudaMemcpyDeviceToHost, h->st), "d2h"));
  OMM_TRY(cuda_status(cudaMemcpyAsync(&ok, dok, sizeof(int), cudaMemcpyDeviceToHost, h->st), "d2h"));
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "sync"));
  *E = out[0];
  if (resid) {
    *resid = ok ? std::sqrt(out[1] / std::max(out[2], 1e-300)) : std::nan("");
    if (resid_orth) *resid_orth = ok ? std::sqrt(out[3]) : std::nan("");
  }
  return OMM_OK;
}

omm_status build_spp(omm_ctx* h) {
  if (!h->spp_built) {
    h->spp = spp_build_structure(h->dim, h->m, h->prm.stencil_radius);
    const SppStructure& s = h->spp;
    int kmax = 0;   // largest right-hand-side block of any product (per-level sizing)
    for (size_t lh = 0; lh < s.fkmax.size(); ++lh) kmax = std::max(kmax, std::max(s.fkmax[lh], s.bkmax[lh]));
    h->trsv_smem = trsv_smem_bytes(h->dbl, kmax, 0);
    if (h->trsv_smem > 220 * 1024) return OMM_EUNSUPPORTED;
    std::vector<int> ns, nb, off, boff, uoff;
    std::vector<long long> wf, wb;
    for (auto& nd : s.nodes) {
      ns.push_back(nd.ns); nb.push_back(nd.nb); off.push_back(nd.off); boff.push_back(nd.boff);
      uoff.push_back(nd.uoff); wf.push_back(nd.wf); wb.push_back(nd.wb);
    }
    OMM_TRY(upload_vec(h, &h->d_node_ns, ns));
    OMM_TRY(upload_vec(h, &h->d_node_nb, nb));
    OMM_TRY(upload_vec(h, &h->d_node_off, off));
    OMM_TRY(upload_vec(h, &h->d_node_boff, boff));
    OMM_TRY(upload_vec(h, &h->d_node_uoff, uoff));
    OMM_TRY(upload_vec(h, &h->d_node_wf, wf));
    OMM_TRY(upload_vec(h, &h->d_node_wb, wb));
    OMM_TRY(upload_vec(h, &h->d_perm, s.perm));
    OMM_TRY(upload_vec(h, &h->d_bnat, s.bnat));
    OMM_TRY(upload_vec(h, &h->d_bnd, s.bnd));
    OMM_TRY(upload_vec(h, &h->d_iperm, s.iperm));
    OMM_TRY(upload_vec(h, &h->d_cptr, s.contrib_ptr));
    OMM_TRY(upload_vec(h, &h->d_cidx, s.contrib_idx));
    OMM_TRY(upload_vec(h, &h->d_fblocks, s.fblocks));
    OMM_TRY(upload_vec(h, &h->d_bblocks, s.bblocks));
    {
      // byte model of the triangular-solve phases (complex elements)
      double nl = 0, ubl = 0, ubs = 0, flv = 0;
      std::vector<char> isleaf(s.nodes.size(), 0);
      for (int id : s.leaf_nodes) isleaf[id] = 1;
      for (size_t id = 0; id < s.nodes.size(); ++id) {
        const SppNode& nd = s.nodes[id];
        if (isleaf[id]) { nl += nd.ns; ubl += nd.nb; }
        else { ubs += nd.nb; flv += 2.0 * (double)(nd.ns + nd.nb) * nd.ns; }
      }
      const double nsep = (double)s.n - nl;
      h->n_leaf = nl;
      h->n_sep = nsep;
      h->tb_leaf_fwd_sys = 2 * nl + ubl;              // b in, y out, update rows out
      h->tb_leaf_bwd_sys = ubl + 2 * nl;              // halo x in, y in, x out
      h->tb_leaf_pole = (double)s.leaf_size;
      h->tb_lvl_sys = nsep + (double)s.contrib_idx.size() + 2 * nsep + nsep + ubs   // forward
                      + nsep + ubs + nsep;                                          // backward
      h->tb_lvl_pole = flv;
    }
    {
      std::vector<int> lunk;
      h->lunk_start.assign(s.levels.size(), 0);
      h->lunk_count.assign(s.levels.size(), 0);
      for (size_t lh = 0; lh < s.levels.size(); ++lh) {
        h->lunk_start[lh] = (int)lunk.size();
        for (int id : s.levels[lh])
          for (int i = 0; i < s.nodes[id].ns; ++i) lunk.push_back(s.nodes[id].off + i);
        h->lunk_count[lh] = (int)lunk.size() - h->lunk_start[lh];
      }
      OMM_TRY(upload_vec(h, &h->d_lunk, lunk));
    }
    OMM_TRY(h->dalloc_t(&h->d_trsv_bar, 4 * sizeof(unsigned)));
    OMM_TRY(cuda_status(cudaMemsetAsync(h->d_trsv_bar, 0, 4 * sizeof(unsigned), h->st), "memset"));
    OMM_TRY(upload_vec(h, &h->d_leaf_nodes, s.leaf_nodes));
    OMM_TRY(upload_vec(h, &h->d_leaf_voff, s.leaf_voff));
    OMM_TRY(upload_vec(h, &h->d_leaf_ioff_bs, s.leaf_ioff_bs));
    OMM_TRY(upload_vec(h, &h->d_leaf_ioff_sb, s.leaf_ioff_sb));
    OMM_TRY(upload_vec(h, &h->d_leaf_bs_idx, s.leaf_bs_idx));
    OMM_TRY(upload_vec(h, &h->d_leaf_sb_idx, s.leaf_sb_idx));
    OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "sync"));
    h->spp_built = true;
  }
  return OMM_OK;
}

}  // namespace

// ======================================================================= C ABI
extern "C" {

const char* omm_strerror(omm_status s) {
  switch (s) {
    case OMM_OK: return "success";
    case OMM_EINVAL: return "invalid argument";
    case OMM_ENOMEM: return "out of memory";
    case OMM_EUNSUPPORTED: return "unsupported grid or option";
    case OMM_ENOTCONV: return "iteration limit reached";
    case OMM_ETIMEOUT: return "device wait timed out";
    case OMM_ECUDA: return "CUDA error";
    case OMM_ESHIFT: return "H - sigma is not negative definite";
    case OMM_ESTATE: return "call out of order";
  }
  return "unknown status";
}

const char* omm_last_error_message(void) { return g_last_error.c_str(); }

omm_status omm_default_params(omm_params* p) {
  if (!p) return OMM_EINVAL;
  p->precision = OMM_FP64;
  p->inner = OMM_INNER_SPARSIFY;
  p->gmres_m = 15;
  p->gmres_cycles = 5;
  p->gmres_rtol = 1e-5;
  p->gmres_fixed = 0;
  p->stencil_radius = 1;
  p->pivot_floor = 1e-12;
  p->tol = 1e-13;
  p->maxit = 50;
  p->refilter = 0;
  p->gram_tensor = 0;
  p->real_orbitals = 0;
  p->trsv_streams = 0;
  p->fixed_iters = 0;
  p->trsv_persistent = 0;
  p->refilter_rtol = 0.0;
  p->gap = 0.0;
  p->launch_overlap = 1;
  p->device_factor = 1;
  return OMM_OK;
}

omm_status omm_default_shift(const omm_grid* g, const double* V, double* shift) {
  if (!g || !V || !shift || (g->dim != 2 && g->dim != 3) || g->m[0] < 2 || !(g->box_len > 0)) return OMM_EINVAL;
  const int m = g->m[0];
  const size_t n = (g->dim == 3) ? (size_t)m * m * m : (size_t)m * m;
  double vmax = V[0], vmin = V[0];
  for (size_t i = 1; i < n; ++i) {
    vmax = std::max(vmax, V[i]);
    vmin = std::min(vmin, V[i]);
  }
  const double tmax = kinetic_max(g->dim, m, g->box_len);
  *shift = tmax + std::max(vmax, 0.0) + 1e-3 * (tmax + vmax - vmin);
  return OMM_OK;
}

omm_status omm_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* ctx) {
  if ((alloc == nullptr) != (release == nullptr)) return OMM_EINVAL;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_alloc = alloc;
  g_free = release;
  g_alloc_ctx = ctx;
  return OMM_OK;
}

omm_status omm_create(const omm_grid* g, const double* V, int N, double shift, const omm_params* p, void* stream,
                      omm_t* out) {
  if (!g || !V || !out) return OMM_EINVAL;
  *out = nullptr;
  if (g->dim != 2 && g->dim != 3) return OMM_EINVAL;
  const int m = g->m[0];
  if (g->m[1] != m || (g->dim == 3 && g->m[2] != m) || !radix_ok(m) || !(g->box_len > 0)) return OMM_EUNSUPPORTED;
  const size_t n = (g->dim == 3) ? (size_t)m * m * m : (size_t)m * m;
  if (N < 1 || (size_t)N >= n) return OMM_EINVAL;
  omm_params prm;
  omm_default_params(&prm);
  if (p) prm = *p;
  if (prm.gmres_m < 1 || prm.gmres_m > 15 || prm.gmres_cycles < 1 || prm.maxit < 0 || prm.refilter < 0 ||
      (prm.precision != OMM_FP64 && prm.precision != OMM_MIXED) || prm.inner < 0 || prm.inner > 2 ||
      prm.trsv_persistent < 0 || prm.trsv_persistent > 1 || prm.launch_overlap < 0 || prm.launch_overlap > 1 ||
      prm.device_factor < 0 || prm.device_factor > 1 ||
      prm.stencil_radius != 1 || prm.trsv_streams < 0 || prm.trsv_streams > omm_ctx::kTrsvStreams ||
      !(prm.gmres_rtol >= 0.0) || !std::isfinite(prm.gmres_rtol) || !(prm.tol >= 0.0) || !std::isfinite(prm.tol) ||
      !(prm.pivot_floor >= 0.0) || !std::isfinite(prm.pivot_floor) || !std::isfinite(shift) || prm.fixed_iters < 0 ||
      !(prm.refilter_rtol >= 0.0) || !std::isfinite(prm.refilter_rtol) || !(prm.gap >= 0.0) || !std::isfinite(prm.gap))
    return OMM_EINVAL;
  const bool dbl = prm.precision == OMM_FP64;
  if (!fused_fft_supported(g->dim, m, dbl) && !big_fft_supported(g->dim, m)) return OMM_EUNSUPPORTED;
  if (!fused_fft_supported(g->dim, m, true) && !big_fft_supported(g->dim, m)) return OMM_EUNSUPPORTED;
  double vmax = V[0];
  for (size_t i = 1; i < n; ++i) vmax = std::max(vmax, V[i]);
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(V[i])) return OMM_EINVAL;
  if (!(shift > kinetic_max(g->dim, m, g->box_len) + vmax)) return OMM_ESHIFT;

  omm_ctx* h = new (std::nothrow) omm_ctx();
  if (!h) return OMM_ENOMEM;
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    h->alloc = g_alloc;
    h->release = g_free;
    h->alloc_ctx = g_alloc_ctx;
  }
  h->dim = g->dim;
  h->m = m;
  h->n = n;
  h->N = N;
  h->L = g->box_len;
  h->shift = shift;
  h->kin = 2.0 * M_PI * M_PI / (g->box_len * g->box_len);
  h->prm = prm;
  h->cur_rtol = prm.gmres_rtol;
  h->dbl = dbl;
  h->csz = dbl ? 16 : 8;
  h->st = (cudaStream_t)stream;
  h->Vh.assign(V, V + n);
  double lm = 0.0;
  for (size_t i = 0; i < n; ++i) lm += V[i];
  h->lmean = lm / n;
  auto fail = [&](omm_status s) { delete h; return s; };
  omm_status s;
  const size_t cnt = (size_t)N * n;
  if ((s = h->dalloc(&h->V, n * (dbl ? 8 : 4))) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->V64, n * 8)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->tw, m * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->tw64, m * 16)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->blk, 4 * cnt * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->Grad, cnt * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->G, cnt * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->Gp, cnt * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc_t(&h->gram, (size_t)2 * N * 4 * N * sizeof(double2))) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->gram_work, std::max(gram_work_bytes(2 * N, 4 * N, n), gram_work_bytes(N, 4 * N, n)))) !=
      OMM_OK)
    return fail(s);
  if ((s = h->dalloc(&h->M1, (size_t)N * N * h->csz)) != OMM_OK) return fail(s);
  if ((s = h->dalloc(&h->M2, (size_t)N * N * h->csz)) != OMM_OK) return fail(s);
  // the CG scalars, then the line search's per-row partial traces (N x 12 doubles)
  const size_t sc_bytes = (sizeof(OmmScalars) + 255) / 256 * 256;
  if ((s = h->dalloc(&h->sc_block, sc_bytes + (size_t)N * 12 * sizeof(double))) != OMM_OK) return fail(s);
  h->sc = (OmmScalars*)h->sc_block;
  h->ls_work = (double*)((char*)h->sc_block + sc_bytes);
  if ((s = h->dalloc(&h->red_work, redot_work_bytes())) != OMM_OK) return fail(s);
  if ((s = h->dalloc_t(&h->shifts, PMAX * sizeof(double2))) != OMM_OK) return fail(s);
  if ((s = h->dalloc_t(&h->zero_shift, sizeof(double2))) != OMM_OK) return fail(s);
  if ((s = h->dalloc_t(&h->wts, PMAX * sizeof(double2))) != OMM_OK) return fail(s);
  if ((s = h->dalloc_t(&h->nact_d, sizeof(int))) != OMM_OK) return fail(s);
  if (cudaMallocHost((void**)&h->sc_h, sizeof(OmmScalars)) != cudaSuccess) return fail(OMM_ENOMEM);
  if (cudaMallocHost((void**)&h->nact_h, sizeof(int)) != cudaSuccess) return fail(OMM_ENOMEM);
  if (dbl)
    s = cuda_status(cudaMemcpyAsync(h->V, V, n * 8, cudaMemcpyHostToDevice, h->st), "V");
  else {
    std::vector<float> vf(V, V + n);
    s = cuda_status(cudaMemcpyAsync(h->V, vf.data(), n * 4, cudaMemcpyHostToDevice, h->st), "V");
    if (s == OMM_OK) s = cuda_status(cudaStreamSynchronize(h->st), "sync");
  }
  if (s != OMM_OK) return fail(s);
  if ((s = cuda_status(cudaMemcpyAsync(h->V64, V, n * 8, cudaMemcpyHostToDevice, h->st), "V64")) != OMM_OK) return fail(s);
  if ((s = upload_twiddles(h, h->tw, dbl)) != OMM_OK) return fail(s);
  if ((s = upload_twiddles(h, h->tw64, true)) != OMM_OK) return fail(s);
  if ((s = cuda_status(cudaMemsetAsync(h->zero_shift, 0, sizeof(double2), h->st), "memset")) != OMM_OK) return fail(s);
  if ((s = cuda_status(cudaMemsetAsync(h->blk, 0, 4 * cnt * h->csz, h->st), "memset")) != OMM_OK) return fail(s);
  if ((s = cuda_status(cudaMemsetAsync(h->sc, 0, sizeof(OmmScalars), h->st), "memset")) != OMM_OK) return fail(s);
  if ((s = cuda_status(cudaStreamSynchronize(h->st), "sync")) != OMM_OK) return fail(s);
  *out = h;
  return OMM_OK;
}

void omm_destroy(omm_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

// Real orbitals: (H - conj z)^-1 R = conj((H - z)^-1 R) for real H and R, so a conjugate
// pair contributes w Y + conj(w Y) = 2 Re(w Y) and one solve of the pair suffices.
// Returns the kept poles (2 w for a pair, w for a real pole) or false if some pole has
// no conjugate partner.
static bool fold_conjugate_pairs(int P, const double* z, const double* w, std::vector<double>& zk,
                                 std::vector<double>& wk) {
  std::vector<char> used(P, 0);
  zk.clear();
  wk.clear();
  auto close = [](double a, double b, double scale) { return std::fabs(a - b) <= 1e-10 * scale; };
  for (int j = 0; j < P; ++j) {
    if (used[j]) continue;
    used[j] = 1;
    const double zs = std::hypot(z[2 * j], z[2 * j + 1]) + 1e-300, ws = std::hypot(w[2 * j], w[2 * j + 1]) + 1e-300;
    if (close(z[2 * j + 1], 0.0, zs) && close(w[2 * j + 1], 0.0, ws)) {   // real pole, real weight
      zk.insert(zk.end(), {z[2 * j], 0.0});
      wk.insert(wk.end(), {w[2 * j], 0.0});
      continue;
    }
    int k = -1;
    for (int t = j + 1; t < P && k < 0; ++t)
      if (!used[t] && close(z[2 * t], z[2 * j], zs) && close(z[2 * t + 1], -z[2 * j + 1], zs) &&
          close(w[2 * t], w[2 * j], ws) && close(w[2 * t + 1], -w[2 * j + 1], ws))
        k = t;
    if (k < 0) return false;
    used[k] = 1;
    zk.insert(zk.end(), {z[2 * j], z[2 * j + 1]});
    wk.insert(wk.end(), {2.0 * w[2 * j], 2.0 * w[2 * j + 1]});
  }
  return true;
}

// Maps of the device factorisation (once per handle); leaves fmaps_ok false when the
// structure does not admit it (then the host factorisation runs).
omm_status ensure_factor_maps(omm_ctx* h) {
  if (h->fmaps_tried) return OMM_OK;
  h->fmaps_tried = true;
  const SppStructure& s = h->spp;
  const SppFactorMaps mp = spp_factor_maps(s);
  if (!mp.ok) return OMM_OK;
  OMM_TRY(upload_vec(h, &h->d_foff, mp.foff));
  OMM_TRY(upload_vec(h, &h->d_child0, mp.child0));
  OMM_TRY(upload_vec(h, &h->d_child1, mp.child1));
  OMM_TRY(upload_vec(h, &h->d_asm_ptr, mp.asm_ptr));
  OMM_TRY(upload_vec(h, &h->d_asm_pos, mp.asm_pos));
  OMM_TRY(upload_vec(h, &h->d_asm_src, mp.asm_src));
  OMM_TRY(upload_vec(h, &h->d_nbr, mp.nbr));
  OMM_TRY(upload_vec(h, &h->d_emap, mp.emap));
  OMM_TRY(upload_vec(h, &h->d_leaf_of, mp.leaf_of));
  OMM_TRY(upload_vec(h, &h->d_Vdbl, h->Vh));
  OMM_TRY(h->dalloc_t(&h->d_qq, (size_t)2 * PMAX * 27 * sizeof(double2)));
  std::vector<int> hn, start;
  h->fheights.clear();
  for (const auto& lev : s.levels) {
    FactorHeight fh;
    start.push_back((int)hn.size());
    fh.count = (int)lev.size();
    int max_ns = 0;
    for (int id : lev) {
      const SppNode& nd = s.nodes[id];
      max_ns = std::max(max_ns, nd.ns);
      fh.max_nf = std::max(fh.max_nf, nd.ns + nd.nb);
      if (mp.leaf_of[id] < 0) {
        fh.dense_nodes = true;
        fh.wprod_tiles = std::max(fh.wprod_tiles, 2 * ((nd.ns + 31) / 32) * ((nd.nb + 31) / 32));
      } else {
        fh.has_leaves = true;
      }
    }
    fh.max_ns = max_ns;
    fh.npanels = (max_ns + 31) / 32;
    if (fh.npanels > FactorHeight::kMaxPanels) return OMM_OK;   // stays with the host factorisation
    for (int q = 0; q < fh.npanels; ++q) {
      int tiles = 0;
      for (int id : lev) {
        const SppNode& nd = s.nodes[id];
        if (q * 32 >= nd.ns) continue;
        const int tm = (nd.ns + nd.nb - std::min(q * 32 + 32, nd.ns) + 31) / 32;
        tiles = std::max(tiles, tm * tm);
      }
      fh.trail_tiles[q] = tiles;
    }
    h->fheights.push_back(fh);
    hn.insert(hn.end(), lev.begin(), lev.end());
  }
  OMM_TRY(upload_vec(h, &h->d_hnodes, hn));
  for (size_t lh = 0; lh < h->fheights.size(); ++lh) h->fheights[lh].nodes = h->d_hnodes + start[lh];
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "maps sync"));
  h->front_size = mp.front_size;
  h->fmaps_ok = true;
  return OMM_OK;
}

// The multifrontal factorisation of P for the P poles of sten on the device, height by
// height, in FP64, into the handle's factor and leaf arrays (rounded once to complex64 for
// a mixed handle); the pivot statistics into spp_poles.  The fronts (and, for a mixed
// handle, the FP64 factor) live in work buffers for the duration of the call.
omm_status device_factor(omm_ctx* h, int P, const std::vector<SppStencil>& sten) {
  const SppStructure& s = h->spp;
  const int na = (int)s.offsets.size() / 3;
  if (na > 27) return OMM_EUNSUPPORTED;
  std::vector<double2> qq((size_t)2 * PMAX * 27, make_double2(0.0, 0.0));
  for (int j = 0; j < P; ++j)
    for (int t = 0; t < na; ++t) {
      qq[(size_t)j * na + t] = make_double2(sten[j].q[t].real(), sten[j].q[t].imag());
      qq[(size_t)PMAX * 27 + (size_t)j * na + t] = make_double2(sten[j].qg[t].real(), sten[j].qg[t].imag());
    }
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->d_qq, qq.data(), qq.size() * sizeof(double2), cudaMemcpyHostToDevice, h->st),
                      "q"));
  const int nn = (int)s.nodes.size();
  const size_t fbytes = (size_t)P * h->front_size * sizeof(double2), pbytes = (size_t)P * nn * 3 * sizeof(double);
  const size_t nfac = (size_t)P * s.factor_size, nleaf = (size_t)P * s.leaf_size;
  const size_t wbytes = h->dbl ? 0 : (nfac + nleaf) * sizeof(double2);
  double2* fronts = nullptr;
  double* pst = nullptr;
  double2* work64 = nullptr;   // mixed handles: the FP64 factor, then the FP64 leaf data
  OMM_TRY(h->dalloc_t(&fronts, fbytes));
  omm_status rc = h->dalloc_t(&pst, pbytes);
  if (rc == OMM_OK && wbytes) rc = h->dalloc_t(&work64, wbytes);
  double2* fac64 = h->dbl ? (double2*)h->factor : work64;
  double2* leaf64 = h->dbl ? (double2*)h->leafvals : work64 + nfac;
  if (rc == OMM_OK) {
    FactorArgs fa;
    fa.node_ns = h->d_node_ns;
    fa.node_nb = h->d_node_nb;
    fa.node_boff = h->d_node_boff;
    fa.node_wf = h->d_node_wf;
    fa.node_wb = h->d_node_wb;
    fa.foff = h->d_foff;
    fa.child0 = h->d_child0;
    fa.child1 = h->d_child1;
    fa.asm_ptr = h->d_asm_ptr;
    fa.asm_pos = h->d_asm_pos;
    fa.asm_src = h->d_asm_src;
    fa.nbr = h->d_nbr;
    fa.emap = h->d_emap;
    fa.leaf_of = h->d_leaf_of;
    fa.leaf_voff = h->d_leaf_voff;
    fa.leaf_ioff_bs = h->d_leaf_ioff_bs;
    fa.leaf_ioff_sb = h->d_leaf_ioff_sb;
    fa.leaf_bs_idx = h->d_leaf_bs_idx;
    fa.leaf_sb_idx = h->d_leaf_sb_idx;
    fa.leaf_bw = s.leaf_bw;
    fa.na = na;
    fa.nnodes = nn;
    fa.front_size = h->front_size;
    fa.factor_size = s.factor_size;
    fa.leaf_size = s.leaf_size;
    fa.V = h->d_Vdbl;
    fa.lmean = sten[0].lmean;
    fa.q = h->d_qq;
    fa.qg = h->d_qq + (size_t)PMAX * 27;
    fa.pivot_floor = h->prm.pivot_floor;
    for (size_t lh = 0; lh < h->fheights.size() && rc == OMM_OK; ++lh)
      rc = cuda_status(launch_factor_height(fa, h->fheights[lh], P, fronts, fac64, leaf64, pst, h->st), "factor");
    if (rc == OMM_OK && !h->dbl)
      rc = cuda_status(launch_factor_to_c64(fac64, (float2*)h->factor, nfac, h->st), "factor c64");
    if (rc == OMM_OK && !h->dbl && nleaf)
      rc = cuda_status(launch_factor_to_c64(leaf64, (float2*)h->leafvals, nleaf, h->st), "leaf c64");
    std::vector<double> ps((size_t)P * nn * 3);
    if (rc == OMM_OK)
      rc = cuda_status(cudaMemcpyAsync(ps.data(), pst, pbytes, cudaMemcpyDeviceToHost, h->st), "pivots");
    if (rc == OMM_OK) rc = cuda_status(cudaStreamSynchronize(h->st), "factor sync");
    if (rc == OMM_OK)
      for (int j = 0; j < P; ++j) {
        SppPole& pp = h->spp_poles[j];
        pp.pivot_min = 1e300;
        pp.pivot_max = 0.0;
        pp.nperturbed = 0;
        for (int id = 0; id < nn; ++id) {
          const double* e = &ps[((size_t)j * nn + id) * 3];
          pp.pivot_min = std::min(pp.pivot_min, e[0]);
          pp.pivot_max = std::max(pp.pivot_max, e[1]);
          pp.nperturbed += (int)e[2];
        }
      }
  }
  cudaStreamSynchronize(h->st);   // the work buffers are idle before they are released
  h->dfree(work64, wbytes);
  h->dfree(pst, pbytes);
  h->dfree(fronts, fbytes);
  return rc;
}

omm_status omm_set_poles(omm_t h, int P, const double* z, const double* w) {
  if (!h || !z || !w || P < 1 || P > PMAX) return OMM_EINVAL;
  for (int j = 0; j < 2 * P; ++j)
    if (!std::isfinite(z[j]) || !std::isfinite(w[j])) return OMM_EINVAL;
  std::vector<double> zf, wf;
  if (h->prm.real_orbitals) {
    if (!fold_conjugate_pairs(P, z, w, zf, wf)) {
      omm_internal_set_message("real_orbitals: a pole has no conjugate partner");
      return OMM_EINVAL;
    }
    P = (int)zf.size() / 2;
    z = zf.data();
    w = wf.data();
  }
  // from here on the handle's pole data changes: it counts as set again only once every
  // buffer below holds the new poles (a failure leaves OMM_ESTATE, not a mix of old and new)
  h->poles_set = false;
  h->real_combine = h->prm.real_orbitals != 0;
  h->use_proj = false;   // a projector built from other poles no longer applies
  h->P = P;
  h->z.resize(P);
  h->w.resize(P);
  std::vector<double2> sh(P);
  for (int j = 0; j < P; ++j) {
    h->z[j] = make_double2(z[2 * j], z[2 * j + 1]);
    h->w[j] = make_double2(w[2 * j], w[2 * j + 1]);
    sh[j] = make_double2(h->shift + z[2 * j], z[2 * j + 1]);
  }
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->shifts, sh.data(), P * sizeof(double2), cudaMemcpyHostToDevice, h->st), "shifts"));
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->wts, h->w.data(), P * sizeof(double2), cudaMemcpyHostToDevice, h->st), "w"));
  OMM_TRY(ensure_gmres_work(h, P));
  const int inner = h->prm.inner;
  if (inner == OMM_INNER_KINETIC || inner == OMM_INNER_SPARSIFY) {
    const size_t n = h->n;
    std::vector<cd> ghat_all(P * n);
    std::vector<cd> q_all;
    if (inner == OMM_INNER_SPARSIFY) {
      OMM_TRY(build_spp(h));
      if (h->prm.device_factor) OMM_TRY(ensure_factor_maps(h));
      const bool dev = h->prm.device_factor && h->fmaps_ok;
      h->spp_poles.assign(P, SppPole());
      std::vector<std::vector<cd>> gh(P);
      std::vector<SppStencil> sten(P);
      // one thread per pole; host cores beyond the poles factor each pole's elimination tree
      // with up to 4 threads (the factor is the same bitwise).  With the device
      // factorisation the host computes only each pole's stencil data (q by the SVD).
      const int hw = std::max(1, (int)std::thread::hardware_concurrency());
      const int nth = std::max(1, std::min<int>(P, hw));
      const int tpp = std::max(1, std::min(4, hw / nth));
      std::vector<std::thread> th;
      for (int t = 0; t < nth; ++t)
        th.emplace_back([&, t]() {
          for (int j = t; j < P; j += nth) {
            if (dev) {
              spp_pole_stencil(h->spp, h->kin, h->Vh.data(), h->shift, cd(z[2 * j], z[2 * j + 1]), sten[j], gh[j]);
              h->spp_poles[j].q = sten[j].q;
              h->spp_poles[j].sigma_min = sten[j].sigma_min;
              h->spp_poles[j].sigma_max = sten[j].sigma_max;
            } else {
              spp_setup_pole(h->spp, h->kin, h->Vh.data(), h->shift, cd(z[2 * j], z[2 * j + 1]), h->prm.pivot_floor,
                             h->spp_poles[j], gh[j], tpp);
            }
          }
        });
      for (auto& t : th) t.join();
      h->nq = (int)h->spp.offsets.size() / 3;
      q_all.resize((size_t)P * h->nq);
      for (int j = 0; j < P; ++j) {
        std::copy(gh[j].begin(), gh[j].end(), ghat_all.begin() + (size_t)j * n);
        std::copy(h->spp_poles[j].q.begin(), h->spp_poles[j].q.end(), q_all.begin() + (size_t)j * h->nq);
      }
      const long long fs = h->spp.factor_size;
      if (h->Pfac < P) {
        h->Pfac = 0;
        OMM_TRY(h->dalloc(&h->factor, (size_t)P * fs * h->csz));
        // (the device factorisation leaves the unused W blocks of 2D leaves as they are)
        OMM_TRY(cuda_status(cudaMemsetAsync(h->factor, 0, (size_t)P * fs * h->csz, h->st), "memset"));
        OMM_TRY(h->dalloc(&h->leafvals, (size_t)P * h->spp.leaf_size * h->csz));
        OMM_TRY(h->dalloc(&h->ubuf, (size_t)h->spp.urows * P * h->N * h->csz));
        OMM_TRY(h->dalloc(&h->ynd, (size_t)P * h->N * n * h->csz));
        OMM_TRY(h->dalloc(&h->xnd, (size_t)P * h->N * n * h->csz));
        // the backward products of systems masked off read xnd entries nothing wrote:
        // keep them finite
        OMM_TRY(cuda_status(cudaMemsetAsync(h->xnd, 0, (size_t)P * h->N * n * h->csz, h->st), "memset"));
        h->Pfac = P;
      }
      h->last_factor_device = dev;
      if (dev) {
        OMM_TRY(device_factor(h, P, sten));
      } else {
        std::vector<cd> fall((size_t)P * fs);
        for (int j = 0; j < P; ++j)
          std::copy(h->spp_poles[j].factor.begin(), h->spp_poles[j].factor.end(), fall.begin() + (size_t)j * fs);
        OMM_TRY(upload_complex(h, h->factor, fall, h->dbl));
        const long long ls = h->spp.leaf_size;
        std::vector<cd> lall((size_t)P * ls);
        for (int j = 0; j < P; ++j)
          std::copy(h->spp_poles[j].leafval.begin(), h->spp_poles[j].leafval.end(), lall.begin() + (size_t)j * ls);
        OMM_TRY(upload_complex(h, h->leafvals, lall, h->dbl));
      }
    } else {
      std::vector<cd> gh;
      for (int j = 0; j < P; ++j) {
        green_symbol(h->dim, h->m, h->kin, h->lmean, h->shift, cd(z[2 * j], z[2 * j + 1]), gh);
        std::copy(gh.begin(), gh.end(), ghat_all.begin() + (size_t)j * n);
      }
      h->nq = 1;
      q_all.assign(P, cd(1.0, 0.0));
    }
    if (!h->ghat_ready) {
      OMM_TRY(h->dalloc(&h->ghat, (size_t)PMAX * n * h->csz));
      OMM_TRY(h->dalloc(&h->qd, (size_t)PMAX * 27 * h->csz));
      h->ghat_ready = true;
    }
    OMM_TRY(upload_complex(h, h->ghat, ghat_all, h->dbl));
    OMM_TRY(upload_complex(h, h->qd, q_all, h->dbl));
  }
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "sync"));
  h->poles_set = true;
  return OMM_OK;
}

omm_status omm_set_orbitals(omm_t h, const void* X) {
  if (!h || !X) return OMM_EINVAL;
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->X(), X, (size_t)h->N * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "set X"));
  if (h->prm.real_orbitals) return cuda_status(launch_real_part(h->dbl, (size_t)h->N * h->n, h->X(), h->st), "real X");
  return OMM_OK;
}

omm_status omm_get_orbitals(omm_t h, void* X) {
  if (!h || !X) return OMM_EINVAL;
  return cuda_status(cudaMemcpyAsync(X, h->X(), (size_t)h->N * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "get X");
}

omm_status omm_filter(omm_t h) {
  if (!h) return OMM_EINVAL;
  if (!h->poles_set) return OMM_ESTATE;
  OMM_TRY(h->use_proj ? apply_projector(h, h->X(), h->G, +1.0) : pole_solve(h, h->X(), h->G, +1.0));
  return cuda_status(cudaMemcpyAsync(h->X(), h->G, (size_t)h->N * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "copy");
}

omm_status omm_iterate(omm_t h, int k, omm_stats* st) {
  if (!h || k < 0) return OMM_EINVAL;
  if (!h->poles_set && !h->use_gtpa) return OMM_ESTATE;
  if (st) std::memset(st, 0, sizeof(*st));
  h->gmres_total = 0;
  int done = 0;
  bool conv = false;
  omm_status s = cg_steps(h, k, st, &done, &conv);
  if (st) {
    st->iters = done;
    st->converged = conv;
  }
  if (s == OMM_OK && h->breakdown) s = OMM_ENOTCONV;
  return s;
}

omm_status omm_solve(omm_t h, omm_stats* st) {
  if (!h) return OMM_EINVAL;
  if (!h->poles_set && !h->use_gtpa) return OMM_ESTATE;
  omm_stats loc;
  std::memset(&loc, 0, sizeof(loc));
  h->gmres_total = 0;
  int total = 0;
  bool conv = false;
  // gTPA is no spectral filter: one CG round from the orbitals as given (Sec. 4's runs
  // of the TPA-type preconditioners start from the initial guess)
  const int rounds = h->use_gtpa ? 0 : h->prm.refilter;
  const int kmax = h->prm.fixed_iters > 0 ? h->prm.fixed_iters : h->prm.maxit;
  omm_status rs = OMM_OK;
  for (int round = 0; round <= rounds; ++round) {
    // the first round at gmres_rtol, the refilter rounds at refilter_rtol
    h->cur_rtol = (round > 0 && h->prm.refilter_rtol > 0.0) ? h->prm.refilter_rtol : h->prm.gmres_rtol;
    if (!h->use_gtpa) {
      rs = omm_filter(h);
      if (rs != OMM_OK) break;
      loc.filters++;
    }
    int done = 0;
    rs = cg_steps(h, kmax, &loc, &done, &conv);
    total += done;
    if (rs != OMM_OK || h->breakdown) break;
  }
  h->cur_rtol = h->prm.gmres_rtol;
  OMM_TRY(rs);
  loc.iters = total;
  loc.converged = conv;
  double E = 0.0, r = 0.0, ro = 0.0;
  omm_status s = energy_fp64(h, &E, &r, &ro);
  if (s == OMM_OK) {
    loc.energy_fp64 = E;
    loc.resid_fp64 = r;
    loc.resid_orth = ro;
    loc.angle_bound = h->prm.gap > 0.0 ? ro / h->prm.gap : 0.0;
  } else if (s != OMM_EUNSUPPORTED) {
    return s;
  }
  if (st) *st = loc;
  return conv ? OMM_OK : OMM_ENOTCONV;
}

omm_status omm_solve_enqueue(omm_t h) {
  if (!h) return OMM_EINVAL;
  if (!h->poles_set && !h->use_gtpa) return OMM_ESTATE;
  if (h->prm.fixed_iters < 1) {
    omm_internal_set_message("omm_solve_enqueue needs fixed_iters > 0 (a fixed CG schedule)");
    return OMM_EINVAL;
  }
  if (!h->fp64_ready || !h->gram || (h->prm.gram_tensor && !h->dbl && !h->tc_err)) {
    omm_internal_set_message("omm_solve_enqueue: call omm_solve once first (it allocates the work space)");
    return OMM_ESTATE;
  }
  h->enqueue_only = true;
  h->gmres_total = 0;
  omm_status s = OMM_OK;
  const int rounds = h->use_gtpa ? 0 : h->prm.refilter;
  for (int round = 0; round <= rounds && s == OMM_OK; ++round) {
    h->cur_rtol = (round > 0 && h->prm.refilter_rtol > 0.0) ? h->prm.refilter_rtol : h->prm.gmres_rtol;
    if (!h->use_gtpa) s = omm_filter(h);
    int done = 0;
    bool conv = false;
    if (s == OMM_OK) s = cg_steps(h, h->prm.fixed_iters, nullptr, &done, &conv);
  }
  if (s == OMM_OK) {
    double E = 0.0, r = 0.0, ro = 0.0;
    s = energy_fp64(h, &E, &r, &ro);
  }
  h->cur_rtol = h->prm.gmres_rtol;
  h->enqueue_only = false;
  h->enqueued = s == OMM_OK;
  return s;
}

omm_status omm_read_result(omm_t h, omm_stats* st) {
  if (!h || !st) return OMM_EINVAL;
  if (!h->enqueued) return OMM_ESTATE;
  std::memset(st, 0, sizeof(*st));
  const int N = h->N;
  const size_t nn = (size_t)N * N;
  const double* dres = (const double*)((double2*)h->m64 + 5 * nn);
  double out[4] = {0.0, 0.0, 0.0, 0.0};
  int ok = 0;
  OMM_TRY(cuda_status(cudaMemcpyAsync(out, dres, sizeof(out), cudaMemcpyDeviceToHost, h->st), "d2h"));
  OMM_TRY(cuda_status(cudaMemcpyAsync(&ok, dres + 4, sizeof(int), cudaMemcpyDeviceToHost, h->st), "d2h"));
  OMM_TRY(read_scalars(h));
  if (!h->use_proj && !h->use_gtpa) OMM_TRY(gmres_stats(h));
  const int rounds = h->use_gtpa ? 0 : h->prm.refilter;
  st->iters = h->prm.fixed_iters * (rounds + 1);
  st->filters = h->use_gtpa ? 0 : rounds + 1;
  st->energy = h->sc_h->E1;
  st->grad_norm = std::sqrt(std::max(h->sc_h->grad2, 0.0));
  st->energy_fp64 = out[0];
  st->resid_fp64 = ok ? std::sqrt(out[1] / std::max(out[2], 1e-300)) : std::nan("");
  st->resid_orth = ok ? std::sqrt(out[3]) : std::nan("");
  st->angle_bound = h->prm.gap > 0.0 ? st->resid_orth / h->prm.gap : 0.0;
  st->gmres_iters_max = h->last_gmres_max;
  st->gmres_relres_max = h->last_relres_max;
  const bool finite = std::isfinite(h->sc_h->E1) && std::isfinite(h->sc_h->t) && std::isfinite(h->sc_h->beta);
  st->converged = finite && !h->sc_h->bad && h->sc_h->converged;
  if (h->sc_h->bad) return OMM_ESHIFT;
  if (!finite) {
    omm_internal_set_message("non-finite energy, line-search step or beta in the CG");
    return OMM_ENOTCONV;
  }
  return OMM_OK;
}

omm_status omm_energy(omm_t h, double* E) {
  if (!h || !E) return OMM_EINVAL;
  return energy_fp64(h, E, nullptr);
}

omm_status omm_apply_h(omm_t h, const void* X, void* Y, int ncols, double s_re, double s_im) {
  if (!h || !X || !Y || ncols < 0) return OMM_EINVAL;
  if (!h->tmp_shift) OMM_TRY(h->dalloc_t(&h->tmp_shift, sizeof(double2) * 2));
  const double2 sh = make_double2(h->shift + s_re, s_im);
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->tmp_shift, &sh, sizeof(sh), cudaMemcpyHostToDevice, h->st), "shift"));
  OMM_TRY(happly(h, X, Y, ncols, h->tmp_shift, ncols > 0 ? ncols : 1, nullptr));
  return cuda_status(cudaStreamSynchronize(h->st), "sync");
}

omm_status omm_gram(omm_t h, const void* A, int na, const void* B, int nb, void* C) {
  if (!h || !A || !B || !C || na < 1 || nb < 1) return OMM_EINVAL;
  OMM_TRY(ensure_dbg_work(h, gram_work_bytes(na, nb, h->n)));
  OMM_TRY(gram_any(h, A, na, B, nb, (double2*)C, nb, h->gw_dbg));
  return read_scalars(h);
}

omm_status omm_gradient(omm_t h, const void* X, void* HX, void* Grad) {
  if (!h || !X || !Grad) return OMM_EINVAL;
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->X(), X, (size_t)h->N * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "X"));
  OMM_TRY(start_cg(h));
  OMM_TRY(cuda_status(
      launch_block_update(h->dbl, h->X(), h->HX(), h->M1, h->M2, 0.0, 2.0, h->N, h->n, Grad, h->st), "grad"));
  if (HX) {
    // (H - sigma) X = H0 X - sigma X
    OMM_TRY(cuda_status(cudaMemcpyAsync(HX, h->HX(), (size_t)h->N * h->n * h->csz, cudaMemcpyDeviceToDevice, h->st), "c"));
    if (!h->tmp_shift) OMM_TRY(h->dalloc_t(&h->tmp_shift, sizeof(double2) * 2));
    const double2 ms[2] = {make_double2(-h->shift, 0.0), make_double2(1.0, 0.0)};
    OMM_TRY(cuda_status(cudaMemcpyAsync(h->tmp_shift, ms, sizeof(ms), cudaMemcpyHostToDevice, h->st), "s"));
    OMM_TRY(cuda_status(launch_axpby(h->dbl, (size_t)h->N * h->n, h->tmp_shift, h->X(), h->tmp_shift + 1, HX, h->st), "ax"));
  }
  return cuda_status(cudaStreamSynchronize(h->st), "sync");
}

omm_status omm_quartic(omm_t h, const void* X, const void* D, double* c, double* t) {
  if (!h || !X || !D) return OMM_EINVAL;
  const size_t cnt = (size_t)h->N * h->n;
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->X(), X, cnt * h->csz, cudaMemcpyDeviceToDevice, h->st), "X"));
  OMM_TRY(cuda_status(cudaMemcpyAsync(h->D(), D, cnt * h->csz, cudaMemcpyDeviceToDevice, h->st), "D"));
  OMM_TRY(happly(h, h->X(), h->HX(), h->N, h->zero_shift, h->N, nullptr));
  OMM_TRY(happly(h, h->D(), h->HD(), h->N, h->zero_shift, h->N, nullptr));
  OMM_TRY(gram_any(h, h->blk, 2 * h->N, h->blk, 4 * h->N, h->gram, 4 * h->N, h->gram_work));
  OMM_TRY(cuda_status(launch_line_search(h->dbl, h->gram, h->N, h->shift, 1, h->prm.tol, h->sc, h->M1, h->M2, h->ls_work, h->st),
                      "ls"));
  OMM_TRY(read_scalars(h));
  if (c)
    for (int i = 0; i < 5; ++i) c[i] = h->sc_h->c[i];
  if (t) *t = h->sc_h->t;
  return h->sc_h->bad ? OMM_ESHIFT : OMM_OK;
}

omm_status omm_precond_apply(omm_t h, int pole, const void* B, void* U, int ncols) {
  if (!h || !B || !U || ncols < 1 || ncols > h->N) return OMM_EINVAL;
  if (!h->poles_set || h->prm.inner != OMM_INNER_SPARSIFY) return OMM_ESTATE;
  if (pole < 0 || pole >= h->P) return OMM_EINVAL;
  // one pole, ncols systems: Green + stencil into the GMRES scratch, then the solves
  const size_t n = h->n;
  OMM_TRY(greenq(h, B, h->tv, ncols, h->nq, ncols, nullptr, (char*)h->ghat + (size_t)pole * n * h->csz,
                 (char*)h->qd + (size_t)pole * h->nq * h->csz, h->d_iperm));
  TrsvArgs a = trsv_args(h, ncols, (size_t)ncols);
  TrsvLevels lv = trsv_levels(h);
  const void* f = (char*)h->factor + (size_t)pole * h->spp.factor_size * h->csz;
  OMM_TRY(cuda_status(launch_spp_solve(SPP_ALL, h->dbl, a, lv, leaf_args(h, pole), 1, h->tv, h->ynd, h->ubuf, U, h->xnd,
                                       f, nullptr, h->trsv_smem, h->prm.launch_overlap, h->st),
                      "spp"));
  return cuda_status(cudaStreamSynchronize(h->st), "sync");
}

omm_status omm_pole_solve(omm_t h, const void* R, void* Y, omm_stats* st) {
  if (!h || !R || !Y) return OMM_EINVAL;
  if (!h->poles_set && !h->use_gtpa) return OMM_ESTATE;
  OMM_TRY(precondition(h, R, Y, 1.0));
  if (!h->use_proj && !h->use_gtpa) OMM_TRY(gmres_stats(h));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    if (!h->use_gtpa) {
      st->gmres_iters_max = h->last_gmres_max;
      st->gmres_relres_max = h->last_relres_max;
    }
  }
  return OMM_OK;
}

// Host Cholesky of the Hermitian positive definite N x N matrix S (row-major FP64) and the
// inverse of its upper factor: S = R^* R, Ri = R^-1.  False if a pivot is not positive.
static bool chol_inverse(const double2* S, int ldS, int N, std::vector<cd>& Ri) {
  std::vector<cd> R((size_t)N * N, cd(0.0, 0.0));
  for (int j = 0; j < N; ++j) {
    double d = S[(size_t)j * ldS + j].x;
    for (int k = 0; k < j; ++k) d -= std::norm(R[(size_t)k * N + j]);
    if (!(d > 0.0)) return false;
    const double rjj = std::sqrt(d);
    R[(size_t)j * N + j] = rjj;
    for (int i = j + 1; i < N; ++i) {
      cd acc(S[(size_t)j * ldS + i].x, S[(size_t)j * ldS + i].y);
      for (int k = 0; k < j; ++k) acc -= std::conj(R[(size_t)k * N + j]) * R[(size_t)k * N + i];
      R[(size_t)j * N + i] = acc / rjj;
    }
  }
  Ri.assign((size_t)N * N, cd(0.0, 0.0));
  for (int c = 0; c < N; ++c) {
    Ri[(size_t)c * N + c] = 1.0 / R[(size_t)c * N + c];
    for (int r = c - 1; r >= 0; --r) {
      cd acc(0.0, 0.0);
      for (int k = r + 1; k <= c; ++k) acc += R[(size_t)r * N + k] * Ri[(size_t)k * N + c];
      Ri[(size_t)r * N + c] = -acc / R[(size_t)r * N + r];
    }
  }
  return true;
}

// Rank-revealing step on the Gram G = Y^* Y of K columns (row-major FP64): Cholesky with
// diagonal pivoting for N steps (the Gram form of QR with column pivoting).  Returns the
// chosen columns piv[0..N) and the K x N coefficient block M (row-major) with
// Y M = Y(:, piv) R11^-1, an orthonormal basis of the chosen columns.
static bool pivoted_select(const std::vector<double2>& Gd, int K, int N, std::vector<int>& piv,
                           std::vector<cd>& M) {
  std::vector<cd> G((size_t)K * K);
  for (size_t e = 0; e < G.size(); ++e) G[e] = cd(Gd[e].x, Gd[e].y);
  piv.resize(K);
  for (int i = 0; i < K; ++i) piv[i] = i;
  std::vector<cd> R((size_t)N * K, cd(0.0, 0.0));   // rows of the pivoted factor (in original column order)
  std::vector<double> dg(K);
  for (int i = 0; i < K; ++i) dg[i] = G[(size_t)i * K + i].real();
  for (int j = 0; j < N; ++j) {
    int best = j;
    for (int i = j + 1; i < K; ++i)
      if (dg[piv[i]] > dg[piv[best]]) best = i;
    std::swap(piv[j], piv[best]);
    const int pj = piv[j];
    if (!(dg[pj] > 0.0)) return false;
    const double rjj = std::sqrt(dg[pj]);
    R[(size_t)j * K + pj] = rjj;
    for (int i = j + 1; i < K; ++i) {
      const int pi = piv[i];
      cd acc = G[(size_t)pj * K + pi];
      for (int k = 0; k < j; ++k) acc -= std::conj(R[(size_t)k * K + pj]) * R[(size_t)k * K + pi];
      R[(size_t)j * K + pi] = acc / rjj;
      dg[pi] -= std::norm(R[(size_t)j * K + pi]);
    }
  }
  // R11 (N x N upper, in pivot order) and its inverse
  std::vector<cd> R11((size_t)N * N, cd(0.0, 0.0)), Ri((size_t)N * N, cd(0.0, 0.0));
  for (int r = 0; r < N; ++r)
    for (int c = r; c < N; ++c) R11[(size_t)r * N + c] = R[(size_t)r * K + piv[c]];
  for (int c = 0; c < N; ++c) {
    Ri[(size_t)c * N + c] = 1.0 / R11[(size_t)c * N + c];
    for (int r = c - 1; r >= 0; --r) {
      cd acc(0.0, 0.0);
      for (int k = r + 1; k <= c; ++k) acc += R11[(size_t)r * N + k] * Ri[(size_t)k * N + c];
      Ri[(size_t)r * N + c] = -acc / R11[(size_t)r * N + r];
    }
  }
  M.assign((size_t)K * N, cd(0.0, 0.0));
  for (int r = 0; r < N; ++r)
    for (int c = 0; c < N; ++c) M[(size_t)piv[r] * N + c] = Ri[(size_t)r * N + c];
  piv.resize(N);
  return true;
}

omm_status omm_build_projector(omm_t h, const void* B, int ncols, omm_stats* st) {
  if (!h || !B) return OMM_EINVAL;
  if (!h->poles_set) return OMM_ESTATE;
  const int N = h->N;
  if (ncols != N && ncols != 2 * N) return OMM_EINVAL;
  const size_t cnt = (size_t)N * h->n;
  if (!h->proj_ready) {
    OMM_TRY(h->dalloc(&h->Uproj, cnt * h->csz));
    OMM_TRY(h->dalloc(&h->projM, (size_t)N * N * h->csz));
    OMM_TRY(h->dalloc(&h->projZero, (size_t)N * N * h->csz));
    OMM_TRY(h->dalloc_t(&h->projC, (size_t)4 * N * N * sizeof(double2)));
    OMM_TRY(cuda_status(cudaMemsetAsync(h->projZero, 0, (size_t)N * N * h->csz, h->st), "memset"));
    // FP64: [Y1 | Y2 | T] blocks, the coefficient blocks and the Gram work
    OMM_TRY(h->dalloc(&h->projY64, 3 * cnt * 16));
    OMM_TRY(h->dalloc(&h->projM64, (size_t)2 * N * N * 16));
    OMM_TRY(h->dalloc(&h->projZero64, (size_t)N * N * 16));
    OMM_TRY(h->dalloc(&h->projWork64, gram_work_bytes(2 * N, 2 * N, h->n)));
    OMM_TRY(cuda_status(cudaMemsetAsync(h->projZero64, 0, (size_t)N * N * 16, h->st), "memset"));
    h->proj_ready = true;
  }
  h->use_proj = false;
  void* Y64 = h->projY64;                      // Y1, then Y2 at + cnt (2N contiguous columns)
  void* T64 = (char*)h->projY64 + 2 * cnt * 16;
  // Y = sum_j w_j (H - sigma - z_j)^-1 B  (Algorithm 2: the pole solves), N columns at a time
  int gmax = 0;
  double rmax = 0.0;
  for (int part = 0; part < ncols / N; ++part) {
    OMM_TRY(pole_solve(h, (const char*)B + part * cnt * h->csz, h->Uproj, 1.0));
    OMM_TRY(gmres_stats(h));
    gmax = std::max(gmax, h->last_gmres_max);
    rmax = std::max(rmax, h->last_relres_max);
    void* dst = (char*)Y64 + part * cnt * 16;
    if (h->dbl)
      OMM_TRY(cuda_status(cudaMemcpyAsync(dst, h->Uproj, cnt * 16, cudaMemcpyDeviceToDevice, h->st), "copy"));
    else
      PROF(PC_VEC, 24.0 * cnt, 1, cuda_status(launch_convert(true, cnt, h->Uproj, dst, h->st), "convert"));
  }
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->gmres_iters_max = gmax;
    st->gmres_relres_max = rmax;
  }
  // Everything below is FP64 (the block, the Grams, the factors and the products): the
  // orthonormal basis U = Y(:, chosen) R^-1 amplifies the rounding of Y by cond(R).
  const int K = ncols;
  std::vector<double2> S((size_t)K * K);
  auto gram64 = [&](int cols) -> omm_status {
    PROF(PC_GRAM, 2.0 * cols * h->n * 16, 2,
         cuda_status(launch_gram(true, Y64, cols, Y64, cols, h->n, h->projC, cols, h->projWork64, h->st), "gram64"));
    OMM_TRY(cuda_status(cudaMemcpyAsync(S.data(), h->projC, (size_t)cols * cols * sizeof(double2),
                                        cudaMemcpyDeviceToHost, h->st),
                        "gram d2h"));
    return cuda_status(cudaStreamSynchronize(h->st), "sync");
  };
  auto apply64 = [&](const std::vector<cd>& Mtop, const std::vector<cd>* Mbot) -> omm_status {
    // T = Y1 Mtop (+ Y2 Mbot), then Y1 = T
    OMM_TRY(cuda_status(cudaMemcpyAsync(h->projM64, Mtop.data(), (size_t)N * N * 16, cudaMemcpyHostToDevice, h->st),
                        "M h2d"));
    void* M2 = h->projZero64;
    const void* Yb = Y64;
    if (Mbot) {
      M2 = (char*)h->projM64 + (size_t)N * N * 16;
      OMM_TRY(cuda_status(cudaMemcpyAsync(M2, Mbot->data(), (size_t)N * N * 16, cudaMemcpyHostToDevice, h->st),
                          "M h2d"));
      Yb = (const char*)Y64 + cnt * 16;
    }
    PROF(PC_BLOCKUPD, (Mbot ? 3.0 : 2.0) * cnt * 16, 1,
         cuda_status(launch_block_update(true, Y64, Yb, h->projM64, M2, 0.0, 0.0, N, h->n, T64, h->st), "qr"));
    OMM_TRY(cuda_status(cudaMemcpyAsync(Y64, T64, cnt * 16, cudaMemcpyDeviceToDevice, h->st), "copy"));
    return cuda_status(cudaStreamSynchronize(h->st), "sync");   // the host vectors are reused
  };
  int passes = 2;   // Cholesky QR passes on N columns
  if (K == 2 * N) {
    // rank-revealing step: the N dominant columns of [Y1 Y2] and their orthonormal basis
    OMM_TRY(gram64(K));
    std::vector<int> piv;
    std::vector<cd> M;
    if (!pivoted_select(S, K, N, piv, M)) {
      omm_internal_set_message("omm_build_projector: the filtered block is rank deficient");
      return OMM_EINVAL;
    }
    std::vector<cd> Mt(M.begin(), M.begin() + (size_t)N * N), Mb(M.begin() + (size_t)N * N, M.end());
    OMM_TRY(apply64(Mt, &Mb));
    passes = 1;   // one more pass restores orthogonality to FP64 rounding
  }
  std::vector<cd> Ri;
  for (int pass = 0; pass < passes; ++pass) {
    OMM_TRY(gram64(N));
    if (!chol_inverse(S.data(), N, N, Ri)) {
      omm_internal_set_message("omm_build_projector: the filtered block is rank deficient");
      return OMM_EINVAL;
    }
    OMM_TRY(apply64(Ri, nullptr));
  }
  if (h->dbl)
    OMM_TRY(cuda_status(cudaMemcpyAsync(h->Uproj, Y64, cnt * 16, cudaMemcpyDeviceToDevice, h->st), "copy"));
  else
    PROF(PC_VEC, 24.0 * cnt, 1, cuda_status(launch_convert(false, cnt, Y64, h->Uproj, h->st), "convert"));
  h->use_proj = true;
  h->use_gtpa = false;
  return OMM_OK;
}

omm_status omm_drop_projector(omm_t h) {
  if (!h) return OMM_EINVAL;
  h->use_proj = false;
  return OMM_OK;
}

omm_status omm_set_gtpa(omm_t h, int t, const double* c, double tau) {
  if (!h || t < 0 || t > 16 || !(tau > 0.0) || !std::isfinite(tau)) return OMM_EINVAL;
  std::vector<double> cc(t + 2);
  if (c) {
    for (int k = 0; k < t + 2; ++k) {
      if (!std::isfinite(c[k]) || c[k] < 0.0) return OMM_EINVAL;
      cc[k] = c[k];
    }
    if (!(cc[0] > 0.0) || !(cc[t + 1] > 0.0)) return OMM_EINVAL;
  } else {
    // c_k = 27 (2/3)^k for k <= t and c_{t+1} = 3 * 27 (2/3)^{t+1}: eq. TPA at t = 3
    for (int k = 0; k <= t; ++k) cc[k] = 27.0 * std::pow(2.0 / 3.0, k);
    cc[t + 1] = 3.0 * 27.0 * std::pow(2.0 / 3.0, t + 1);
  }
  const size_t n = h->n;
  const int m = h->m;
  h->use_gtpa = false;   // set again once the new table is on the device
  std::vector<cd> tab(2 * n);
  auto sk = [m](int i) { return i < m / 2 ? i : i - m; };
  for (size_t i = 0; i < n; ++i) {
    const int ix = (int)(i % m), iy = (int)((i / m) % m), iz = h->dim == 3 ? (int)(i / ((size_t)m * m)) : 0;
    const double k2 = (double)sk(ix) * sk(ix) + (double)sk(iy) * sk(iy) + (h->dim == 3 ? (double)sk(iz) * sk(iz) : 0.0);
    const double s = k2 / tau;
    double p = cc[t], st = s;            // Horner for p_t(s); s^{t+1} alongside
    for (int k = t - 1; k >= 0; --k) {
      p = p * s + cc[k];
      st *= s;
    }
    double g = p / (p + cc[t + 1] * st);
    if (!std::isfinite(g)) g = 0.0;      // s^{t+1} and p_t both overflowed: the limit s -> inf
    tab[i] = cd(g / (double)n, 0.0);
    tab[n + i] = cd(-g / (double)n, 0.0);
  }
  if (!h->gtpa_one) {
    void* one = nullptr;
    OMM_TRY(h->dalloc(&one, h->csz));
    OMM_TRY(upload_complex(h, one, std::vector<cd>(1, cd(1.0, 0.0)), h->dbl));
    h->gtpa_one = one;
  }
  if (!h->gtpa_tab) OMM_TRY(h->dalloc(&h->gtpa_tab, 2 * n * h->csz));
  OMM_TRY(upload_complex(h, h->gtpa_tab, tab, h->dbl));
  OMM_TRY(cuda_status(cudaStreamSynchronize(h->st), "gtpa sync"));
  h->use_gtpa = true;
  return OMM_OK;
}

omm_status omm_drop_gtpa(omm_t h) {
  if (!h) return OMM_EINVAL;
  h->use_gtpa = false;
  return OMM_OK;
}

omm_status omm_factor_info(omm_t h, int pole, int* nsuper, long long* nnz, double* pivot_ratio, int* nperturbed) {
  if (!h) return OMM_EINVAL;
  if (!h->poles_set || h->prm.inner != OMM_INNER_SPARSIFY) return OMM_ESTATE;
  if (pole < 0 || pole >= h->P) return OMM_EINVAL;
  const SppPole& pp = h->spp_poles[pole];
  if (nsuper) *nsuper = (int)h->spp.nodes.size();
  if (nnz) *nnz = h->spp.factor_size;
  if (pivot_ratio) *pivot_ratio = pp.pivot_max > 0 ? pp.pivot_min / pp.pivot_max : 0.0;
  if (nperturbed) *nperturbed = pp.nperturbed;
  return OMM_OK;
}

omm_status omm_profile_enable(omm_t h, int on) {
  if (!h || on < 0 || on > 2) return OMM_EINVAL;
  h->prof_flush();
  if (on) {
    for (int c = 0; c < PC_NCLS; ++c) {
      h->prof.ms[c] = 0.0;
      h->prof.calls[c] = 0;
      h->prof.kernels[c] = 0;
      h->prof.bytes[c] = 0.0;
      h->prof.impl_bytes[c] = 0.0;
      h->prof.flops[c] = 0.0;
    }
  }
  h->prof.on = on == 1;
  return OMM_OK;
}

omm_status omm_profile_read_flops(omm_t h, int cls, double* flops) {
  if (!h || !flops || cls < 0 || cls >= PC_NCLS) return OMM_EINVAL;
  *flops = h->prof.flops[cls];
  return OMM_OK;
}

omm_status omm_profile_read_impl(omm_t h, int cls, double* impl_bytes) {
  if (!h || !impl_bytes || cls < 0 || cls >= PC_NCLS) return OMM_EINVAL;
  *impl_bytes = h->prof.impl_bytes[cls];
  return OMM_OK;
}

omm_status omm_profile_read(omm_t h, int cls, long long* calls, long long* kernels, double* ms, double* bytes) {
  if (!h || cls < 0 || cls >= PC_NCLS) return OMM_EINVAL;
  h->prof_flush();
  if (calls) *calls = h->prof.calls[cls];
  if (kernels) *kernels = h->prof.kernels[cls];
  if (ms) *ms = h->prof.ms[cls];
  if (bytes) *bytes = h->prof.bytes[cls];
  return OMM_OK;
}

const char* omm_profile_class_name(int cls) { return (cls >= 0 && cls < PC_NCLS) ? kProfNames[cls] : nullptr; }

omm_status omm_device_bytes(omm_t h, size_t* bytes) {
  if (!h || !bytes) return OMM_EINVAL;
  *bytes = h->bytes;
  return OMM_OK;
}

}  // extern "C"
