// HODLR likelihood engine: context, workspace plan, build / factor / solve / trace
// orchestration and the C ABI of include/hodlr.h.
//
// Data layout (device, column-major panels with leading dimension N, tree order):
//   F[l]     N x cap  level-l factors: rows of left children hold Q (W), rows of right
//                     children hold B~ (X), so the pair block is Q B~^T (eq. lowrnkB11).
//   dF[j][l] N x cap  derivative factors [dQ; dB~] of parameter j (eq. diff low-rank); the
//                     derivative block is dQ B~^T + Q dB~^T (rank 2w).
//   U[l]     N x w_l  K~_{c1}^{-1} W and K~_{c2}^{-1} X of the factorization (App. C), all levels
//            side by side in one buffer.
//   CP[l]    per node (2w x 2w): C^{-1} P with C = [[I, Sx],[Sw, I]] the SMW core of the
//            node (Sw = W^T K~_{c1}^{-1} W, Sx = X^T K~_{c2}^{-1} X) and P the half swap.
//   leaves   A_b, A_b^{-1} (n_l x n_l), dA_b per derivative parameter.
// A node v with children c1, c2 factors as K~_v = diag(K~_c1, K~_c2)(I + U V^T) with
// U = [[W~,0],[0,X~]], V = [[0,W],[X,0]] (eq. one way factor, App. C), so
//   K~_v^{-1} = (I - U C^{-1} V^T) diag(K~_c1^{-1}, K~_c2^{-1}),
//   log|K~_v| = log|K~_c1| + log|K~_c2| + log|I - Lw^T Sx Lw|  (Sw = Lw Lw^T, Sylvester).
// The exact traces of App. B are taken through the same node recursion:
//   tr(K~^{-1} M) = sum_leaves tr(A_b^{-1} M_b) - sum_nodes tr(CP_v U_v^T M_v U_v),
// and the four-factor trace adds, per node, the cross term of the two off-diagonal blocks
// and the C^{-1} corrections (see traces()).
#include <math.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <string>
#include <atomic>
#include <map>
#include <mutex>
#include <memory>
#include <new>
#include <vector>

#include "../../include/hodlr.h"
#include "common.cuh"
#include "ops.h"

namespace hodlr {

// ------------------------------------------------------------------------------ arena
struct Arena {
  char* base = nullptr;
  size_t cap = 0, off = 0;
  bool plan = true;
  template <class X> X* take(size_t n) {
    size_t bytes = ((n * sizeof(X) + 255) / 256) * 256;
    size_t o = off;
    off += bytes;
    if (plan) return nullptr;
    if (off > cap) throw Error(HODLR_ENOMEM, "workspace too small");
    return (X*)(base + o);
  }
};

struct Base {
  virtual ~Base() {}
  std::string err;
  virtual void build(const double* theta) = 0;
  virtual void eval(const double* theta, const double* y, double* nll, double* grad, double* fisher) = 0;
  virtual void apply_nat(const double* theta, int which, const double* X, double* Y, int ncols) = 0;
  virtual void probe(int level, int ncols, double* out) = 0;
  virtual void densify(int which, double* out) = 0;
  virtual void solve_nat(const double* b, double* x) = 0;
  virtual void matvec_nat(int which, const double* X, double* Y, int ncols) = 0;
  virtual void grad_adjoint(const double* y, double* g) = 0;
  virtual void traces(double* t, double* f) = 0;
  virtual void set_pivots(const int32_t* piv) = 0;
  virtual void logdet_levels(double* out) = 0;
  virtual void debug_level(int what, int level, double* out, int64_t count, int32_t* w_out) = 0;
  virtual void get_pivots(int32_t* piv) const = 0;
  virtual void read_perm(int64_t* perm) = 0;   // real tree position -> natural index, from the device maps
  virtual cudaStream_t stream() const = 0;
  // Capture-safe evaluation (NLL and gradient) for CUDA-graph batching: no host
  // synchronisation, static level widths (the rank cap), statuses left on the device; the
  // results land in out() = {nll, g[0..3], status} once the captured work has run.
  virtual void set_stream(cudaStream_t s) = 0;
  // digit-slice tensor-core products for this context's FP64 GEMMs (HODLR_MIXED_BF16): set on
  // entry to every call on the calling thread, cleared on exit
  virtual void oz_enter(bool on) = 0;
  virtual void set_graph_mode(bool on) = 0;
  virtual void eval_graph(const double* theta, const double* y) = 0;
  virtual const double* graph_out() const = 0;
  uint64_t serial = 0;                       // unique per context (graph cache keys)
  bool tune = false;                         // tile autotuner on for this context's products
  bool uses_slices = false;                  // HODLR_MIXED_BF16 context
  // N: rows of the (padded) tree layout; Nr: rows of K (natural order).  An uneven cluster
  // tree (median splits of a size that is not leaf x 2^tau) is laid out with every leaf in a
  // slot of the largest leaf's size: the real rows of a leaf come first in its slot, the rest
  // are padding rows, which every panel keeps at zero and K~ keeps decoupled (unit diagonal).
  int N = 0, Nr = 0, tau = 0, leaf = 0, c = 0, cap = 0, nleaves = 0;
  int npad = 0;                              // padding rows (N - Nr)
  TreeDesc td{};                             // cluster tree (the order itself is made on the device)
  std::vector<int> leafreal;                 // real rows per leaf slot
  // real tree position -> natural index (Nr), by the closed forms of the tree order on the host
  // (planning query only: an engine's device maps come from the tree_order kernel)
  void plan_perm(int64_t* perm) const {
    for (int p = 0; p < td.Ns; ++p) {
      const int s = tree_spatial_pos(td, p);
      int lo, hi;
      tree_leaf(td, s, lo, hi);
      for (int v = 0; v < td.nvar; ++v) perm[td.nvar * lo + v * (hi - lo) + (s - lo)] = (int64_t)v * td.Ns + p;
    }
  }
  std::vector<std::vector<int>> host_rank;   // per level
  long long napply = 0;
  double logdet = 0.0;
  bool built = false;
};

static const int NPAR = 4;  // sigma2, ell, kappa, tau2

template <class T>
struct Engine : Base {
  using Acc = T;
  // model / options
  int dim, G, nvar, prec;
  double nu, tol, guard;
  uint64_t seed;
  int Ns;
  PhysicsDesc ph;
  cudaStream_t st;
  cudaStream_t stream() const override { return st; }
  void set_stream(cudaStream_t s) override { st = s; }
  bool oz = false;                       // HODLR_MIXED_BF16
  Scratch ozwork, ozsplit;
  void oz_enter(bool on) override {
    g_oz_cfg.on = on && oz;
    g_oz_cfg.tune = on && oz && tune && !graph_mode;
    g_oz_cfg.work = on && oz ? ozwork : Scratch{};
    g_oz_cfg.split = on && oz ? ozsplit : Scratch{};
  }
  bool graph_mode = false;
  // entering or leaving graph mode invalidates the build: the host copies of the log-det and
  // the level widths are not refreshed by captured work
  void set_graph_mode(bool on) override { graph_mode = on; built = false; }
  // tree
  std::vector<std::vector<int>> bnd;     // per depth: node boundaries (2^d + 1)
  int* d_perm_plain = nullptr;           // tree-layout row -> natural index (-1 = padding)
  int* d_real2pad = nullptr;             // real tree position -> tree-layout row
  int* d_rowid = nullptr;                // tree-layout row -> real tree position (uneven trees only)
  int* d_leafreal = nullptr;             // real rows per leaf slot
  std::vector<unsigned char*> d_mask;    // per level (1..tau): right-child rows
  // level data
  std::vector<T*> F, CP, dF[2];
  std::vector<double*> U, CP64;        // FP64 factorization data (App. C)
  std::vector<int*> d_rank, d_piv;
  std::vector<double*> d_nodelog;
  std::vector<int> w;                    // width per level
  // leaves
  T *A = nullptr, *Ainv = nullptr, *dA[2] = {nullptr, nullptr};
  double* leaflog = nullptr;
  // physics state (one set per arithmetic type)
  template <class V> struct Phys {
    V *lam0 = nullptr, *lam1 = nullptr, *tw = nullptr, *S = nullptr;
    void* fftw = nullptr;
    size_t fftw_bytes = 0;
    int qc = 0;                            // physics column chunk
    int* perm = nullptr;                   // tree position -> natural index (var-major chunk layout)
    V *nx = nullptr, *na = nullptr, *nb = nullptr, *nu = nullptr, *nu2 = nullptr, *ns = nullptr, *ne = nullptr,
      *nt = nullptr, *nw = nullptr;
    int df = 0;                            // 2-D DST products with double-float accumulation
    float *Shi = nullptr, *Slo = nullptr;  // TF32 split of the FP32 DST matrix (tensor-core products)
    float2 *Sdf = nullptr, *Xdf = nullptr; // double-float split of the DST matrix and a field panel
  };
  Phys<T> P;                               // working precision
  Phys<double> P64;                        // FP64-class leaf sketch of the mixed path
  double* coef = nullptr;                  // Thomas tables (shared)
  float* coef32 = nullptr;                 // FP32 copy of the 2-D tables (FP32 fields)
  // sketch buffers
  T *R = nullptr, *KR = nullptr, *KjR[2] = {nullptr, nullptr}, *Y = nullptr, *S = nullptr, *KS = nullptr,
    *KjS[2] = {nullptr, nullptr}, *dS = nullptr, *KdS = nullptr, *YJ = nullptr, *Q1 = nullptr;
  double *gram = nullptr, *pwork = nullptr;
  T *RinvJ = nullptr, *Rinv = nullptr, *Linv_T = nullptr, *sm1 = nullptr, *sm2 = nullptr, *sm3 = nullptr;
  // factor workspaces (FP64 small)
  double *sw = nullptr, *sx = nullptr, *lw = nullptr, *t1 = nullptr, *t2 = nullptr, *t3 = nullptr, *phi = nullptr;
  // panels for leaves / solves / traces
  T *E[3] = {nullptr, nullptr, nullptr};
  T *WP = nullptr, *WZ = nullptr;       // wide panels N x 10 cap
  T *fg = nullptr, *stb = nullptr;      // solve coefficient blocks
  T *nodeG = nullptr, *nodeX = nullptr; // per-node 2w x 2w matrices
  T *tpan = nullptr;                    // peel T blocks
  double *vec_d = nullptr, *vec_d2 = nullptr, *vec_d3 = nullptr, *red = nullptr, *res = nullptr;
  T* vec_t = nullptr;
  double* Afp = nullptr;                // FP64 leaf blocks, then their Cholesky factors
  double *sgbuf = nullptr, *fg64 = nullptr, *stb64 = nullptr;
  double* Ucat = nullptr;               // factor panels of all levels, side by side
  int q64max = 0;                        // column chunk of the FP64 Woodbury corrections
  int* d_status = nullptr;
  Scratch scratch;
  // state
  double theta_built[4] = {0, 0, 0, 0};
  bool frozen = false;
  int nwide = 10, wide = 0;
  double* LinvLeaf = nullptr;
  double* Ainv64 = nullptr;             // mixed path: leaf inverses for the factorization sweeps (FP64,
                                        // then split in place into double-float pairs)

  Engine(const hodlr_model* m, const hodlr_opts* o, cudaStream_t s_) {
    dim = m->dim; G = m->grid[0]; nvar = m->nvar; nu = m->nu; prec = m->precision;
    oz = prec == HODLR_MIXED_BF16 && sizeof(T) == 8;
    uses_slices = oz;
    leaf = o->leaf; cap = o->rank_or_cap; c = o->rank_or_cap + o->oversample; tol = o->tol; seed = o->seed;
    guard = o->guard > 0.0 ? o->guard : 1e-5;
    st = s_;
    if (dim < 1 || dim > 2 || nvar < 1 || nvar > 2 || G < 2 || leaf < nvar || leaf % nvar || cap < 1 || c < cap ||
        (nu != 0.5 && nu != 1.5))
      throw Error(HODLR_EINVAL, "bad model or options");
    if (dim == 2 && m->grid[1] != G) throw Error(HODLR_EINVAL, "2-D grids must be square");
    Ns = dim == 1 ? G : G * G;
    Nr = nvar * Ns;
    // tree (Sec. 3.2.2 index sets; KD / Morton order of Sec. 5.2): every node [lo, hi) of spatial
    // positions splits at lo + (hi - lo) / 2, tau times
    int lps = leaf / nvar;
    tau = 0;
    while ((Ns + (1 << tau) - 1) / (1 << tau) > lps) ++tau;
    std::vector<std::vector<int>> sb(tau + 1);
    sb[0] = {0, Ns};
    for (int d = 1; d <= tau; ++d) {
      for (size_t q = 0; q + 1 < sb[d - 1].size(); ++q) {
        int lo = sb[d - 1][q], hi = sb[d - 1][q + 1];
        sb[d].push_back(lo);
        sb[d].push_back(lo + (hi - lo) / 2);
      }
      sb[d].push_back(Ns);
    }
    nleaves = 1 << tau;
    // tree layout: leaf slots of the largest leaf's size (padding rows at the end of a slot)
    int slot = 0;
    for (int b = 0; b < nleaves; ++b) slot = std::max(slot, sb[tau][b + 1] - sb[tau][b]);
    this->leaf = nvar * slot;
    N = this->leaf * nleaves;
    npad = N - Nr;
    bnd.assign(tau + 1, {});
    for (int d = 0; d <= tau; ++d)
      for (int q = 0; q <= (1 << d); ++q) bnd[d].push_back((q << (tau - d)) * this->leaf);
    for (int b = 0; b < nleaves; ++b) leafreal.push_back(nvar * (sb[tau][b + 1] - sb[tau][b]));
    td.dim = dim; td.G = G; td.nvar = nvar; td.Ns = Ns; td.tau = tau; td.slot = this->leaf;
    // physics geometry
    ph.dim = dim; ph.G = G; ph.nvar = nvar; ph.nu = nu; ph.h = 1.0 / (G + 1);
    ph.df_fft = oz ? 1 : 0;   // HODLR_MIXED_BF16: FFT butterflies of the FP64 fields in double-float
    int L = 1;
    while (L < 2 * G - 1) L <<= 1;
    ph.L = L; ph.L1 = 0; ph.L2 = 0;
    if (dim == 1 && L > 4096) { ph.L2 = 2048; ph.L1 = L / 2048; }
    if (dim == 2 && L > 4096) throw Error(HODLR_ENOTIMPL, "2-D grids above 2048 points per axis are not built");
    w.assign(tau + 1, 0);
    host_rank.assign(tau + 1, {});
  }

  int npairs(int l) const { return 1 << (l - 1); }
  int msize(int d) const { return bnd[d][1] - bnd[d][0]; }  // node size at depth d

  static T* plan_or(T* base, size_t off) { return base ? base + off : nullptr; }

  template <class V> void carve_phys(Arena& ar, Phys<V>& Q, int qc) {
    qc += qc & 1;
    Q.qc = qc;
    size_t nemb = dim == 1 ? ph.L : (size_t)ph.L * ph.L;
    Q.perm = ar.take<int>(N);
    Q.lam0 = ar.take<V>(nemb);
    Q.lam1 = ar.take<V>(nemb);
    Q.tw = ar.take<V>(2 * (size_t)ph.L + 16);
    if (dim == 2) Q.S = ar.take<V>((size_t)G * G);
    if (dim == 2 && sizeof(V) == 4 && tf32x3_supported(G, G, G, G, G)) {
      Q.Shi = ar.take<float>((size_t)G * G);
      Q.Slo = ar.take<float>((size_t)G * G);
    }
    if (dim == 2 && sizeof(V) == 8 && sizeof(T) == 4) {   // the FP64-class fields of the mixed path
      Q.Sdf = ar.take<float2>((size_t)G * G);
      Q.Xdf = ar.take<float2>((size_t)Ns * qc);
    }
    Q.fftw_bytes = std::max(fft_work_bytes(ph, qc, sizeof(V)), nemb * (sizeof(V) * 3) + 512);
    Q.fftw = ar.take<char>(Q.fftw_bytes);
    size_t nat = (size_t)nvar * Ns * qc;
    Q.nx = ar.take<V>(nat); Q.na = ar.take<V>(nat); Q.nb = ar.take<V>(nat); Q.nu = ar.take<V>(nat);
    Q.nu2 = ar.take<V>(nat); Q.ns = ar.take<V>(nat); Q.ne = ar.take<V>(nat); Q.nt = ar.take<V>(nat);
    Q.nw = ar.take<V>(nat);
  }

  // ---------------------------------------------------------------- workspace plan / carve
  void carve(Arena& ar) {
    const size_t NN = (size_t)N;
    d_perm_plain = ar.take<int>(N);
    d_real2pad = ar.take<int>(Nr);
    d_rowid = npad ? ar.take<int>(N) : nullptr;
    d_leafreal = ar.take<int>(nleaves);
    d_mask.assign(tau + 1, nullptr);
    for (int l = 1; l <= tau; ++l) d_mask[l] = ar.take<unsigned char>(N);
    F.assign(tau + 1, nullptr); U.assign(tau + 1, nullptr); CP.assign(tau + 1, nullptr); CP64.assign(tau + 1, nullptr);
    dF[0].assign(tau + 1, nullptr); dF[1].assign(tau + 1, nullptr);
    d_rank.assign(tau + 1, nullptr); d_piv.assign(tau + 1, nullptr); d_nodelog.assign(tau + 1, nullptr);
    for (int l = 1; l <= tau; ++l) {
      F[l] = ar.take<T>(NN * cap);
      dF[0][l] = ar.take<T>(NN * cap);
      dF[1][l] = ar.take<T>(NN * cap);
      CP[l] = ar.take<T>((size_t)npairs(l) * 4 * cap * cap);
      CP64[l] = ar.take<double>((size_t)npairs(l) * 4 * cap * cap);
      d_rank[l] = ar.take<int>(npairs(l));
      d_piv[l] = ar.take<int>((size_t)npairs(l) * c);
      d_nodelog[l] = ar.take<double>(npairs(l));
    }
    size_t nl2 = (size_t)nleaves * leaf * leaf;
    A = ar.take<T>(nl2);
    Ainv = ar.take<T>(nl2);
    dA[0] = ar.take<T>(nl2);
    dA[1] = ar.take<T>(nl2);
    leaflog = ar.take<double>(nleaves);
    // physics
    carve_phys(ar, P, std::min(64, std::max(c, 2)));
    if (sizeof(T) == 4) { carve_phys(ar, P64, 16); P64.df = 1; }
    coef = ar.take<double>(dim == 1 ? 2 * (size_t)G : 2 * (size_t)G * G);
    if (sizeof(T) == 4 && dim == 2) coef32 = ar.take<float>(2 * (size_t)G * G);
    // sketch
    R = ar.take<T>(NN * c); KR = ar.take<T>(NN * c); KjR[0] = ar.take<T>(NN * c); KjR[1] = ar.take<T>(NN * c);
    Y = ar.take<T>(NN * c);
    S = ar.take<T>(NN * cap); KS = ar.take<T>(NN * cap); KjS[0] = ar.take<T>(NN * cap);
    KjS[1] = ar.take<T>(NN * cap); dS = ar.take<T>(NN * cap); KdS = ar.take<T>(NN * cap);
    YJ = ar.take<T>(NN * cap); Q1 = ar.take<T>(NN * cap);
    int maxp = std::max(1, npairs(std::max(tau, 1)));
    gram = ar.take<double>((size_t)maxp * c * c);
    pwork = ar.take<double>((size_t)maxp * 2 * c * c);
    RinvJ = ar.take<T>((size_t)maxp * cap * cap);
    Rinv = ar.take<T>((size_t)maxp * cap * cap);
    Linv_T = ar.take<T>((size_t)maxp * cap * cap);
    sm1 = ar.take<T>((size_t)maxp * cap * cap);
    sm2 = ar.take<T>((size_t)maxp * cap * cap);
    sm3 = ar.take<T>((size_t)maxp * cap * cap);
    int maxb = 2 * maxp;  // child blocks at the finest level
    sw = ar.take<double>((size_t)maxb * cap * cap);
    sx = ar.take<double>((size_t)maxp * cap * cap);
    lw = ar.take<double>((size_t)maxp * cap * cap);
    t1 = ar.take<double>((size_t)maxp * cap * cap);
    t2 = ar.take<double>((size_t)maxp * cap * cap);
    t3 = ar.take<double>((size_t)maxp * cap * cap);
    phi = ar.take<double>((size_t)maxp * cap * cap);
    // leaves / wide panels
    wide = std::max(nwide * cap, 3 * leaf);
    WP = ar.take<T>(NN * wide);
    WZ = ar.take<T>(NN * wide);
    LinvLeaf = ar.take<double>(nl2);
    if (sizeof(T) == 4) Ainv64 = ar.take<double>(nl2);
    for (int k = 0; k < 3; ++k) E[k] = plan_or(WZ, (size_t)k * NN * leaf);
    size_t qmax = (size_t)wide;
    qmax = std::max<size_t>(qmax, (size_t)c);
    fg = ar.take<T>((size_t)maxb * cap * qmax);
    stb = ar.take<T>((size_t)maxb * cap * qmax);
    tpan = ar.take<T>((size_t)maxb * 2 * ((cap + 3) & ~3) * qmax);   // leading dimension w_l rounded up to 4
    nodeG = ar.take<T>((size_t)maxp * 4 * cap * cap * 12);
    nodeX = ar.take<T>((size_t)maxp * 4 * cap * cap * 8);
    vec_d = ar.take<double>(NN * 2);
    vec_d2 = ar.take<double>(NN * 2);
    vec_d3 = ar.take<double>(NN * 2);
    vec_t = ar.take<T>(NN * 2);
    red = ar.take<double>((size_t)std::max(maxb, nleaves) * 16 + 64);
    res = ar.take<double>(256 + 64);
    Afp = ar.take<double>(nl2);
    sgbuf = ar.take<double>((size_t)maxb * cap * cap);
    q64max = std::max(1, 4 * cap);
    fg64 = ar.take<double>((size_t)maxb * cap * q64max);
    stb64 = ar.take<double>((size_t)maxb * cap * q64max);
    Ucat = ar.take<double>(NN * (size_t)std::max(tau, 1) * cap);
    for (int l = 1; l <= tau; ++l) U[l] = Ucat + NN * (size_t)cap * (l - 1);
    d_status = ar.take<int>(8);
    if (oz) {
      // slice planes for one wide panel (six BF16 digits per FP64 value), at least 256 MB and
      // at most 2 GiB; split-K partials of the long-K products
      size_t ob = (size_t)14 * NN * std::max(wide, c) + ((size_t)1 << 26);
      ob = std::min<size_t>(std::max<size_t>(ob, (size_t)1 << 28), (size_t)1 << 31);
      ozwork.ptr = ar.take<char>(ob);
      ozwork.bytes = ob;
      ozsplit.bytes = (size_t)1 << 28;
      ozsplit.ptr = ar.take<char>(ozsplit.bytes);
    }
    size_t sbytes = std::max<size_t>(64u << 20, (size_t)4 * c * c * 8 * 640);
    scratch.ptr = ar.take<char>(sbytes);
    scratch.bytes = sbytes;
  }

  void upload_tree() {
    tree_order(td, N, d_perm_plain, d_rowid, d_real2pad, st);
    HODLR_CUDA(cudaMemcpyAsync(d_leafreal, leafreal.data(), nleaves * sizeof(int), cudaMemcpyHostToDevice, st));
    upload_phys(P);
    if (P64.perm) upload_phys(P64);
    for (int l = 1; l <= tau; ++l) tree_level_mask(N, msize(l), d_rowid, d_mask[l], st);
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  template <class V> void upload_phys(Phys<V>& Q) {
    tree_phys_perm(d_perm_plain, N, Ns, nvar, Q.qc, Q.perm, st);
    if (dim == 2) dst_matrix<V>(G, Q.S, st);
    if (Q.Shi) tf32_split((const float*)Q.S, Q.Shi, Q.Slo, (long long)G * G, st);
    if (Q.Sdf) df_split((const double*)Q.S, Q.Sdf, (long long)G * G, st);
    if (ph.L1 == 0) twiddles<V>(ph.L, Q.tw, st);
    else {
      twiddles<V>(ph.L1, Q.tw, st);
      twiddles<V>(ph.L2, Q.tw + (ph.L1 / 2) * 2, st);
    }
    HODLR_CUDA(cudaStreamSynchronize(st));
  }

  void status_check(const char* what) {
    if (graph_mode) return;   // left in d_status, read after the captured work has run
    int s = 0;
    HODLR_CUDA(cudaMemcpyAsync(&s, d_status, sizeof(int), cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
    if (s != 0) {
      HODLR_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), st));
      throw Error(s, std::string(what) + ": a Cholesky factorization failed (K~ not SPD)");
    }
  }

  // Products whose accuracy must exceed the digit-slice products' (Gram matrices, whose small
  // eigenvalues carry the rank decisions and the SMW cores): FP64 FMA even on HODLR_MIXED_BF16
  struct FP64Only {
    bool saved;
    FP64Only() : saved(g_oz_cfg.on) { g_oz_cfg.on = false; }
    ~FP64Only() { g_oz_cfg.on = saved; }
  };
  // ---------------------------------------------------------------- GEMM helpers
  void gemmT(GemmArgs g) { gemm<T, T, T, T>(g, scratch, st); }
  // per child block b at depth d: C_b (P x Q) = op(A[b])^T B[b]  (A, B row panels)
  void block_tn(int d, int P, int Qn, const T* Ap, const T* Bp, long long ldb, T* C, long long ldc, long long sC,
                double alpha = 1.0, double beta = 0.0) {
    GemmArgs g;
    int m = msize(d);
    g.M = P; g.N = Qn; g.K = m;
    g.A = Ap; g.lda = N; g.sA = m; g.tA = 1;
    g.B = Bp; g.ldb = ldb; g.sB = m;
    g.C = C; g.ldc = ldc; g.sC = sC;
    g.alpha = alpha; g.beta = beta; g.batch = 1 << d;
    gemmT(g);
  }

  // out -= sum over levels in [l0, l1] of H_l X (or dH^(j)_l X) ; X, out: N x q row panels
  void offdiag(int l0, int l1, int j, const T* X, long long ldx, int q, T* out, long long ldo, double sign = -1.0) {
    offdiag_t<T>(l0, l1, j, X, ldx, q, out, ldo, sign);
  }
  // GEMM with a factor panel (type T) and V panels: V == T in working precision, V = double with
  // double-float accumulation in the mixed path
  template <class V> void fgemm(const GemmArgs& g) {
    if constexpr (std::is_same<V, T>::value) gemm<T, T, T, T>(g, scratch, st);
    else gemm_df<T, V, V>(g, scratch, st);
  }
  template <class V>
  void offdiag_t(int l0, int l1, int j, const V* X, long long ldx, int q, V* out, long long ldo, double sign = -1.0) {
    for (int l = l0; l <= l1; ++l) {
      int wl = w[l];
      if (wl == 0 || q == 0) continue;
      int m = msize(l);
      int nbk = 1 << l;
      // wl x q blocks with the leading dimension rounded up to 4 (16-byte rows for TMA)
      const int wl4 = (wl + 3) & ~3;
      V* tp = (V*)tpan;
      V* tp2 = tp + (size_t)nbk * wl4 * q;
      auto tn = [&](const T* Fp, V* C) {   // C_b = F[b]^T X[b]  (wl x q per child block)
        GemmArgs g;
        g.M = wl; g.N = q; g.K = m;
        g.A = Fp; g.lda = N; g.sA = m; g.tA = 1;
        g.B = X; g.ldb = ldx; g.sB = m;
        g.C = C; g.ldc = wl4; g.sC = (long long)wl4 * q; g.batch = nbk;
        fgemm<V>(g);
      };
      auto nn = [&](const T* Fp, const V* Bp) {   // out[b] += sign F[b] C_{b^1}
        GemmArgs g;
        g.M = m; g.N = q; g.K = wl;
        g.A = Fp; g.lda = N; g.sA = m;
        g.B = Bp; g.ldb = wl4; g.sB = (long long)wl4 * q; g.bmap = BMAP_XOR1;
        g.C = out; g.ldc = ldo; g.sC = m;
        g.alpha = sign; g.beta = 1.0; g.batch = nbk;
        fgemm<V>(g);
      };
      if (j < 0) {
        tn(F[l], tp);
        nn(F[l], tp);
      } else {
        tn(F[l], tp);
        tn(dF[j][l], tp2);
        nn(dF[j][l], tp);   // dQ (B~^T x2) and dB~ (Q^T x1)
        nn(F[l], tp2);      // Q (dB~^T x2) and B~ (dQ^T x1)
      }
    }
  }

  // ---------------------------------------------------------------- physics product
  const double* th = theta_built;
  void set_physics(const double* theta) {
    if (P64.perm) {
      // mixed path: the FP32 spectra are the FP64 ones rounded (same transform order)
      matern_spectra<double>(ph, theta[0], theta[1], P64.lam0, P64.lam1, P64.fftw, P64.tw, st);
      const long long nemb = dim == 1 ? ph.L : (long long)ph.L * ph.L;
      convert<double, T>(P64.lam0, P.lam0, nemb, st);
      convert<double, T>(P64.lam1, P.lam1, nemb, st);
    } else {
      matern_spectra<T>(ph, theta[0], theta[1], P.lam0, P.lam1, P.fftw, P.tw, st);
    }
    tridiag_tables(ph, theta[2], coef, st);
    if (coef32) convert<double, float>(coef, coef32, 2LL * G * G, st);
  }
  template <class V> void Ainv_nat(Phys<V>& Q, const V* in, V* out, int q) {
    DstSplit tc;
    tc.hi = Q.Shi;
    tc.lo = Q.Slo;
    tc.df_S = Q.Sdf;
    tc.df_X = Q.Xdf;
    solve_A<V>(ph, q, in, Ns, out, Ns, coef, Q.S, Q.nw, scratch, st, Q.df,
               std::is_same<V, float>::value ? coef32 : nullptr, tc);
  }
  // K X, K_ell X, K_kappa X on a tree-order panel (q columns); any output may be null
  void apply(const T* X, long long ldx, int q, T* oK, T* oL, T* oKap, long long ldo) {
    apply_t<T>(P, X, ldx, q, oK, oL, oKap, ldo);
  }
  template <class V>
  void apply_t(Phys<V>& Q, const V* X, long long ldx, int q, V* oK, V* oL, V* oKap, long long ldo) {
    const double kap = th[2], t2 = th[3];
    const int qc = Q.qc;
    const size_t vs = (size_t)Ns * qc;   // variable stride in natural buffers
    for (int c0 = 0; c0 < q; c0 += qc) {
      int qq = std::min(qc, q - c0);
      const V* Xc = X + (size_t)c0 * ldx;
      permute_rows<V, V>(Xc, ldx, Q.nx, Ns, Q.perm, N, qq, 1, st);
      auto out = [&](V* dst, const V* src) {
        if (dst) permute_rows<V, V>(src, Ns, dst + (size_t)c0 * ldo, ldo, Q.perm, N, qq, 0, st);
      };
      if (nvar == 1) {
        Ainv_nat(Q, Q.nx, Q.na, qq);                                        // a = A^{-1} x
        if (oKap) Ainv_nat(Q, Q.na, Q.nb, qq);                              // b = A^{-2} x
        if (oK || oKap || oL)
          fft_convolve<V>(ph, qq, Q.na, Ns, Q.lam0, oL ? Q.lam1 : nullptr, Q.nu, Q.nu2, Ns, Q.fftw, Q.tw, st);
        if (oKap) fft_convolve<V>(ph, qq, Q.nb, Ns, Q.lam0, nullptr, Q.ns, nullptr, Ns, Q.fftw, Q.tw, st);
        if (oK || oKap) Ainv_nat(Q, Q.nu, Q.ne, qq);                        // e = A^{-1} K_u a
        if (oK) {
          out(oK, Q.ne);
          axpby<V>(N, qq, t2, Xc, ldx, 1.0, oK + (size_t)c0 * ldo, ldo, st);
        }
        if (oL) {
          Ainv_nat(Q, Q.nu2, Q.nt, qq);
          out(oL, Q.nt);
        }
        if (oKap) {
          axpby<V>(Ns, qq, 1.0, Q.ns, Ns, 1.0, Q.ne, Ns, st);               // e + K_u b
          Ainv_nat(Q, Q.ne, Q.nt, qq);
          axpby<V>(Ns, qq, 0.0, Q.nt, Ns, -2.0 * kap, Q.nt, Ns, st);
          out(oKap, Q.nt);
        }
      } else {
        V* x1 = Q.nx;
        V* x2 = Q.nx + vs;
        V* a = Q.na;
        V* wv = Q.na + vs;
        Ainv_nat(Q, x2, a, qq);                                             // a = A^{-1} x2
        axpby<V>(Ns, qq, 1.0, x1, Ns, 0.0, wv, Ns, st);
        axpby<V>(Ns, qq, 1.0, a, Ns, 1.0, wv, Ns, st);                      // w = x1 + a  (L^T x)
        V* u = Q.nu;       // [u; c1]
        V* u2 = Q.nu2;     // [u'; c2]
        V* s = Q.ns;       // [s; c3]
        if (oK || oKap || oL)
          fft_convolve<V>(ph, qq, wv, Ns, Q.lam0, oL ? Q.lam1 : nullptr, u, u2, Ns, Q.fftw, Q.tw, st);
        if (oK || oKap) Ainv_nat(Q, u, u + vs, qq);                         // c1 = A^{-1} u
        if (oK) {
          out(oK, u);
          axpby<V>(N, qq, t2, Xc, ldx, 1.0, oK + (size_t)c0 * ldo, ldo, st);
        }
        if (oL) {
          Ainv_nat(Q, u2, u2 + vs, qq);
          out(oL, u2);
        }
        if (oKap) {
          V* b = Q.nb;
          Ainv_nat(Q, a, b, qq);                                            // b = A^{-2} x2
          fft_convolve<V>(ph, qq, b, Ns, Q.lam0, nullptr, s, nullptr, Ns, Q.fftw, Q.tw, st);   // s = K_u b
          axpby<V>(Ns, qq, 1.0, u + vs, Ns, 0.0, Q.nt, Ns, st);
          axpby<V>(Ns, qq, 1.0, s, Ns, 1.0, Q.nt, Ns, st);                  // c1 + s
          Ainv_nat(Q, Q.nt, s + vs, qq);                                    // c3
          axpby<V>(Ns, qq, 0.0, s, Ns, -2.0 * kap, s, Ns, st);              // -2 kappa [s; c3]
          axpby<V>(Ns, qq, 0.0, s + vs, Ns, -2.0 * kap, s + vs, Ns, st);
          out(oKap, s);
        }
      }
      napply += (long long)qq * ((oK ? 1 : 0) + (oL ? 1 : 0) + (oKap ? 1 : 0));
    }
  }

  // ---------------------------------------------------------------- build (Alg. 1, Sec. 3.2.2, Alg. 2, Sec. 3.3)
  void build(const double* theta) override {
    for (int k = 0; k < 4; ++k) {
      if (!(theta[k] > 0.0) || !std::isfinite(theta[k])) throw Error(HODLR_EINVAL, "theta must be positive and finite");
      theta_built[k] = theta[k];
    }
    built = false;
    napply = 0;
    HODLR_CUDA(cudaMemsetAsync(d_status, 0, 8 * sizeof(int), st));
    set_physics(theta);
    const double thr = std::max(tol, guard);
    for (int l = 1; l <= tau; ++l) {
      const int np = npairs(l);
      const int m = msize(l);          // child block size
      // --- sketch of the level's blocks: Y = (K - sum_{l'<l} H^(l')) R^(l)
      probe_panel<T>(N, c, l, 0, seed, d_mask[l], d_rowid, R, N, st);
      apply(R, N, c, KR, KjR[0], KjR[1], N);
      HODLR_CUDA(cudaMemcpyAsync(Y, KR, sizeof(T) * (size_t)N * c, cudaMemcpyDeviceToDevice, st));
      offdiag(1, l - 1, -1, R, N, c, Y, N);
      // --- pivoted QR of each left-child block of Y via its FP64 Gram (Alg. 1 step 3)
      {
        GemmArgs g;
        g.M = c; g.N = c; g.K = m;
        g.A = Y; g.lda = N; g.sA = 2 * m; g.tA = 1;
        g.B = Y; g.ldb = N; g.sB = 2 * m;
        g.C = gram; g.ldc = c; g.sC = (long long)c * c; g.batch = np;
        FP64Only exact;
        g64<T, T>(g);
      }
      pivoted_cholesky<T>(np, c, cap, cap, gram, thr, d_rank[l], d_piv[l], RinvJ, frozen ? 1 : 0, pwork, d_status, st);
      status_check("frozen pivots");
      int wl = 0;
      if (graph_mode) {
        // static width: the rank cap (columns beyond a pair's own rank stay zero), so that the
        // captured work does not depend on a value read back from the device
        host_rank[l].assign(np, cap);
        wl = cap;
      } else {
        host_rank[l].resize(np);
        HODLR_CUDA(cudaMemcpyAsync(host_rank[l].data(), d_rank[l], np * sizeof(int), cudaMemcpyDeviceToHost, st));
        HODLR_CUDA(cudaStreamSynchronize(st));
        for (int r : host_rank[l]) wl = std::max(wl, r);
      }
      w[l] = wl;
      fill<T>(F[l], T(0), (long long)N * cap, st);
      fill<T>(dF[0][l], T(0), (long long)N * cap, st);
      fill<T>(dF[1][l], T(0), (long long)N * cap, st);
      if (wl == 0) continue;
      // --- Q = Y_J R_J^{-1}, re-orthogonalised once (CholQR on the FP64 Gram)
      gather_columns<T>(np, m, 2LL * m, Y, N, d_piv[l], c, d_rank[l], wl, YJ, N, st);
      pair_nn(l, wl, YJ, RinvJ, cap, Q1, 1.0, 0.0);
      {
        GemmArgs g;
        g.M = wl; g.N = wl; g.K = m;
        g.A = Q1; g.lda = N; g.sA = 2 * m; g.tA = 1;
        g.B = Q1; g.ldb = N; g.sB = 2 * m;
        g.C = gram; g.ldc = wl; g.sC = (long long)wl * wl; g.batch = np;
        FP64Only exact;
        g64<T, T>(g);
      }
      potrf_lower(np, wl, gram, wl, (long long)wl * wl, d_rank[l], nullptr, d_status, st);
      trtri_lower(np, wl, gram, wl, (long long)wl * wl, t1, st);
      convert<double, T>(t1, Linv_T, (long long)np * wl * wl, st);
      status_check("CholQR");
      // Q = Q1 Linv^T into the left-child rows of F[l]
      {
        GemmArgs g;
        g.M = m; g.N = wl; g.K = wl;
        g.A = Q1; g.lda = N; g.sA = 2 * m;
        g.B = Linv_T; g.ldb = wl; g.sB = (long long)wl * wl; g.tB = 1;
        g.C = F[l]; g.ldc = N; g.sC = 2 * m; g.batch = np;
        gemmT(g);
      }
      // R^{-1} of Y_J = Q R:  RinvJ * Linv^T   (wl x wl per pair)
      {
        GemmArgs g;
        g.M = wl; g.N = wl; g.K = wl;
        g.A = RinvJ; g.lda = cap; g.sA = (long long)cap * cap;
        g.B = Linv_T; g.ldb = wl; g.sB = (long long)wl * wl; g.tB = 1;
        g.C = Rinv; g.ldc = wl; g.sC = (long long)wl * wl; g.batch = np;
        gemmT(g);
      }
      // --- projection: Z = (K - sum H) S^(l), S = [Q; 0];  B~ = Z[c2]
      HODLR_CUDA(cudaMemcpyAsync(S, F[l], sizeof(T) * (size_t)N * wl, cudaMemcpyDeviceToDevice, st));
      apply(S, N, wl, KS, KjS[0], KjS[1], N);
      offdiag(1, l - 1, -1, S, N, wl, KS, N);
      copy_rows_c2(l, wl, KS, F[l]);
      // --- derivatives (Sec. 3.3) for ell (j=0) and kappa (j=1)
      for (int j = 0; j < 2; ++j) {
        T* dY = KjR[j];
        offdiag(1, l - 1, j, R, N, c, dY, N);                              // dY = K_j R - sum dH R
        gather_columns<T>(np, m, 2LL * m, dY, N, d_piv[l], c, d_rank[l], wl, YJ, N, st);
        // Alg. 2 step 1: Y' = Q^T dY R^{-1}
        {
          GemmArgs g;
          g.M = wl; g.N = wl; g.K = m;
          g.A = F[l]; g.lda = N; g.sA = 2 * m; g.tA = 1;
          g.B = YJ; g.ldb = N; g.sB = 2 * m;
          g.C = sm1; g.ldc = wl; g.sC = (long long)wl * wl; g.batch = np;
          gemmT(g);
        }
        small_nn(np, wl, sm1, Rinv, sm2);                                  // Y' = (Q^T dY) R^{-1}
        alg2_core<T>(np, wl, sm2, sm3, st);                                    // step 2: M2 = dOmega - Y'
        // step 3: dQ = dY R^{-1} + Q M2 = Q dOmega + (I - Q Q^T) dY R^{-1}
        pair_nn(l, wl, YJ, Rinv, wl, dF[j][l], 1.0, 0.0);
        pair_nn(l, wl, F[l], sm3, wl, dF[j][l], 1.0, 1.0);
        // dZ = (K_j - sum dH) S + (K - sum H) dS,  dS = [dQ; 0]
        HODLR_CUDA(cudaMemcpyAsync(dS, dF[j][l], sizeof(T) * (size_t)N * wl, cudaMemcpyDeviceToDevice, st));
        apply(dS, N, wl, KdS, nullptr, nullptr, N);
        offdiag(1, l - 1, -1, dS, N, wl, KdS, N);
        T* dZ = KjS[j];
        offdiag(1, l - 1, j, S, N, wl, dZ, N);
        axpby<T>(N, wl, 1.0, KdS, N, 1.0, dZ, N, st);
        copy_rows_c2(l, wl, dZ, dF[j][l]);
      }
    }
    build_leaves();
    factor();
    if (!graph_mode && tc_status_take(st))
      throw Error(HODLR_ETIMEOUT, "a tensor-core product gave up waiting for its operands");
    for (int k = 0; k < 4; ++k) theta_built[k] = theta[k];
    built = true;
  }

  // C[c1 rows of pair p] = alpha * A[c1 rows of p] * B_p + beta * C   (m x wl, B_p: wl x wl, ld ldb)
  void pair_nn(int l, int wl, const T* Ap, const T* Bp, int ldb, T* Cp, double alpha, double beta) {
    int m = msize(l);
    GemmArgs g;
    g.M = m; g.N = wl; g.K = wl;
    g.A = Ap; g.lda = N; g.sA = 2 * m;
    g.B = Bp; g.ldb = ldb; g.sB = (long long)ldb * ldb;
    g.C = Cp; g.ldc = N; g.sC = 2 * m;
    g.alpha = alpha; g.beta = beta; g.batch = npairs(l);
    if (ldb != wl) g.sB = (long long)ldb * ldb;
    gemmT(g);
  }
  void small_nn(int nb, int n, const T* Ap, const T* Bp, T* Cp) {
    GemmArgs g;
    g.M = n; g.N = n; g.K = n;
    g.A = Ap; g.lda = n; g.sA = (long long)n * n;
    g.B = Bp; g.ldb = n; g.sB = (long long)n * n;
    g.C = Cp; g.ldc = n; g.sC = (long long)n * n; g.batch = nb;
    gemmT(g);
  }
  // copy the right-child rows of src (N x wl) into dst, keeping only the first rank_p columns of
  // pair p (B~ = Z[c2, :r]): the shared sketch panel carries other pairs' columns beyond r_p
  void copy_rows_c2(int l, int wl, const T* src, T* dst) {
    int m = msize(l);
    copy_blocks<T, T>(npairs(l), m, wl, src + m, N, 2LL * m, dst + m, N, 2LL * m, 1.0, st);
    zero_pad_cols(l, wl, dst + m);
  }
  void zero_pad_cols(int l, int wl, T* rows);

  // ---------------------------------------------------------------- leaves (eq. leaf sample, eq. diag diff)
  void build_leaves() {
    const int nl = leaf;
    if (sizeof(T) == 4) {
      build_leaves_hp();
    } else {
      // S_leaf = stacked identities
      T* Sl = WP;  // N x nl
      fill<T>(Sl, T(0), (long long)N * nl, st);
      identity_blocks(Sl);
      apply(Sl, N, nl, E[0], E[1], E[2], N);
      offdiag(1, tau, -1, Sl, N, nl, E[0], N);
      offdiag(1, tau, 0, Sl, N, nl, E[1], N);
      offdiag(1, tau, 1, Sl, N, nl, E[2], N);
      extract_leaves<T, double>(nleaves, nl, d_leafreal, E[0], N, Afp, 1.0, st);
      extract_leaves<T, T>(nleaves, nl, d_leafreal, E[1], N, dA[0], 0.0, st);
      extract_leaves<T, T>(nleaves, nl, d_leafreal, E[2], N, dA[1], 0.0, st);
    }
    convert<double, T>(Afp, A, (long long)nleaves * nl * nl, st);
    // FP64 leaf Cholesky, log-det and inverse
    potrf_lower(nleaves, nl, Afp, nl, (long long)nl * nl, nullptr, leaflog, d_status, st);
    double* Linv = LinvLeaf;
    leaf_trtri(Linv);
    {
      GemmArgs g;  // A^{-1} = L^{-T} L^{-1}
      g.M = nl; g.N = nl; g.K = nl;
      g.A = Linv; g.lda = nl; g.sA = (long long)nl * nl; g.tA = 1;
      g.B = Linv; g.ldb = nl; g.sB = (long long)nl * nl;
      g.C = Ainv; g.ldc = nl; g.sC = (long long)nl * nl; g.batch = nleaves;
      if constexpr (sizeof(T) == 8) {
        gemm<double, double, T, double>(g, scratch, st);
      } else {
        g.C = Ainv64;
        gemm_df<double, double, double>(g, scratch, st);
        convert<double, T>(Ainv64, Ainv, (long long)nleaves * nl * nl, st);
        // the leaf solves read it as a double-float operand: split once, in place
        df_split(Ainv64, (float2*)Ainv64, (long long)nleaves * nl * nl, st);
      }
    }
    status_check("leaf Cholesky");
  }
  // L^{-1} of the leaf Cholesky factors by block recursion: the 32 x 32 diagonal blocks are
  // inverted directly, then pairs of blocks of size s merge into 2s with
  //   [[L11, 0], [L21, L22]]^{-1} = [[X11, 0], [-X22 L21 X11, X22]]
  // (two batched products per pair; FP64 on the FP64 path, double-float on the mixed path).
  void leaf_trtri(double* X) {
    const int n = leaf;
    const long long n2 = (long long)n * n;
    if (n < 64 || (n & (n - 1)) != 0) {
      trtri_lower(nleaves, n, Afp, n, n2, X, st);
      return;
    }
    fill<double>(X, 0.0, nleaves * n2, st);
    trtri_diag32(nleaves, n, Afp, n, n2, X, st);
    double* Tm = (double*)WP;    // nleaves x (n/2)^2 products of the merge step
    for (int s = 32; s < n; s *= 2) {
      for (int o = 0; o < n; o += 2 * s) {
        GemmArgs g;   // T = L21 X11
        g.M = s; g.N = s; g.K = s;
        g.A = Afp + (o + s) + (size_t)o * n; g.lda = n; g.sA = n2;
        g.B = X + o + (size_t)o * n; g.ldb = n; g.sB = n2;
        g.C = Tm; g.ldc = s; g.sC = (long long)s * s; g.batch = nleaves;
        g64<double, double>(g);
        GemmArgs h;   // X21 = -X22 T
        h.M = s; h.N = s; h.K = s;
        h.A = X + (o + s) + (size_t)(o + s) * n; h.lda = n; h.sA = n2;
        h.B = Tm; h.ldb = s; h.sB = (long long)s * s;
        h.C = X + (o + s) + (size_t)o * n; h.ldc = n; h.sC = n2;
        h.alpha = -1.0; h.batch = nleaves;
        g64<double, double>(h);
      }
    }
  }
  // Leaf sketch of the mixed path at FP64-class accuracy: the stacked-identity probe makes each
  // leaf entry a difference of two row sums over all leaves (eq. leaf sample), whose FP32
  // rounding would exceed the nugget; the products run in FP64 (FFT, Thomas recurrences, DST
  // with double-float accumulation) and the peeling in double-float, in column chunks.
  void build_leaves_hp() {
    const int nl = leaf;
    // derivative leaves dA_j in working precision (they do not decide positive definiteness)
    {
      T* Sl = WP;
      fill<T>(Sl, T(0), (long long)N * nl, st);
      identity_blocks(Sl);
      apply(Sl, N, nl, nullptr, E[1], E[2], N);
      offdiag(1, tau, 0, Sl, N, nl, E[1], N);
      offdiag(1, tau, 1, Sl, N, nl, E[2], N);
      extract_leaves<T, T>(nleaves, nl, d_leafreal, E[1], N, dA[0], 0.0, st);
      extract_leaves<T, T>(nleaves, nl, d_leafreal, E[2], N, dA[1], 0.0, st);
    }
    // leaf blocks of K~ in FP64-class arithmetic, in column chunks
    const int qcl = std::max(1, std::min(64, wide / 4));
    double* Sx = (double*)WP;
    double* Eh = Sx + (size_t)N * qcl;
    for (int j0 = 0; j0 < nl; j0 += qcl) {
      int qq = std::min(qcl, nl - j0);
      fill<double>(Sx, 0.0, (long long)N * qq, st);
      identity_cols(Sx, j0, qq);
      apply_t<double>(P64, Sx, N, qq, Eh, nullptr, nullptr, N);
      offdiag_t<double>(1, tau, -1, Sx, N, qq, Eh, N);
      scatter_leaf_cols<double, double>(Eh, j0, qq, Afp);
    }
    symmetrize_blocks<double>(Afp);
  }
  void identity_cols(double* Sx, int j0, int qq);
  template <class TS, class TD> void scatter_leaf_cols(const TS* E, int j0, int qq, TD* Ablk);
  template <class V> void symmetrize_blocks(V* Ablk);
  void identity_blocks(T* Sl);

  // ---------------------------------------------------------------- factorization (App. C)
  // solve with the block-diagonal of the depth-d subtrees:  out = diag_v(K~_v^{-1}) in
  void solve_depth(const T* in, long long ldi, T* out, long long ldo, int q, int d) {
    const int nl = leaf;
    if (sizeof(T) == 8 && !(oz && g_oz_cfg.on)) {
      leaf_trsm<T, T>(nleaves, nl, Afp, in, ldi, out, ldo, q, st);      // FP64: backward-stable leaf solves
    } else {
      GemmArgs g;                                                      // FP32 bulk: explicit A_b^{-1}
      g.M = nl; g.N = q; g.K = nl;
      g.A = Ainv; g.lda = nl; g.sA = (long long)nl * nl;
      g.B = in; g.ldb = ldi; g.sB = nl;
      g.C = out; g.ldc = ldo; g.sC = nl; g.batch = nleaves;
      gemmT(g);
    }
    for (int l = tau; l > d; --l) {
      int wl = w[l];
      if (wl == 0) continue;
      int m = msize(l), np = npairs(l), nbk = 1 << l;
      // FG^T_b = out[b]^T F[b]   (q x wl per child block, consecutive -> per pair q x 2wl = [g f]^T)
      GemmArgs g;
      g.M = q; g.N = wl; g.K = m;
      g.A = out; g.lda = ldo; g.sA = m; g.tA = 1;
      g.B = F[l]; g.ldb = N; g.sB = m;
      g.C = fg; g.ldc = q; g.sC = (long long)q * wl; g.batch = nbk;
      gemmT(g);
      // ST^T_p = FG^T_p (CP_p)^T, CP = C^{-1} P  ->  ST = C^{-1} [f; g] = [s; t]
      GemmArgs h;
      h.M = q; h.N = 2 * wl; h.K = 2 * wl;
      h.A = fg; h.lda = q; h.sA = 2LL * q * wl;
      h.B = CP[l]; h.ldb = 2 * wl; h.sB = 4LL * wl * wl; h.tB = 1;
      h.C = stb; h.ldc = q; h.sC = 2LL * q * wl; h.batch = np;
      gemmT(h);
      // out[b] -= U[b] (ST^T_b)^T ; ST^T_b is the b-th q x wl block (s for c1, t for c2)
      GemmArgs k;
      k.M = m; k.N = q; k.K = wl;
      // the FP64 panel in working precision (the sketch buffer Q1 is free during the traces), so
      // that the update runs as a plain working-precision product
      const T* Ul = (const T*)U[l];
      if constexpr (sizeof(T) == 4) {
        convert<double, T>(U[l], Q1, (long long)N * wl, st);
        Ul = Q1;
      }
      k.A = Ul; k.lda = N; k.sA = m;
      k.B = stb; k.ldb = q; k.sB = (long long)q * wl; k.tB = 1;
      k.C = out; k.ldc = ldo; k.sC = m;
      k.alpha = -1.0; k.beta = 1.0; k.batch = nbk;
      gemmT(k);
    }
  }

  // FP64-accurate contraction with FP64 output: plain FP64 (DFMA) on the FP64 path, double-float
  // accumulation on the FP32 pipes on the mixed path (GB300's FP64 rate is low).
  template <class TA, class TB> void g64(const GemmArgs& g) {
    if constexpr (sizeof(T) == 8) gemm<TA, TB, double, double>(g, scratch, st);
    else gemm_df<TA, TB, double>(g, scratch, st);
  }

  // FP64-class solve with the depth-d subtrees (factorization sweeps and K~^{-1} y): leaf solves
  // and Woodbury corrections against the stored factors F (App. C).  The FP64 path solves the
  // leaves by substitution with their Cholesky factors (backward stable); the mixed path
  // applies the FP64 leaf inverses with double-float accumulation, whose error (unit roundoff
  // x cond(A_b), ~1e-10) is far inside that path's accuracy.
  void solve64(const double* in, long long ldi, double* out, long long ldo, int q, int d) {
    leaf_solve64(in, ldi, out, ldo, q);
    for (int l = tau; l > d; --l) woodbury64(l, out, ldo, q);
  }
  void leaf_solve64(const double* in, long long ldi, double* out, long long ldo, int q) {
    if constexpr (sizeof(T) == 8) {
      if (oz && g_oz_cfg.on) {
        // HODLR_MIXED_BF16: the FP64 leaf inverses applied as digit-slice products (error
        // ~ slicing accuracy x cond(A_b)); the FP64 path keeps the backward-stable substitution
        GemmArgs g;
        g.M = leaf; g.N = q; g.K = leaf;
        g.A = Ainv; g.lda = leaf; g.sA = (long long)leaf * leaf;
        g.B = in; g.ldb = ldi; g.sB = leaf;
        g.C = out; g.ldc = ldo; g.sC = leaf; g.batch = nleaves;
        gemm<double, double, double, double>(g, scratch, st);
        return;
      }
      leaf_trsm<double, double>(nleaves, leaf, Afp, in, ldi, out, ldo, q, st);
    } else {
      GemmArgs g;
      g.M = leaf; g.N = q; g.K = leaf;
      g.A = (const float2*)Ainv64; g.lda = leaf; g.sA = (long long)leaf * leaf;
      g.B = in; g.ldb = ldi; g.sB = leaf;
      g.C = out; g.ldc = ldo; g.sC = leaf; g.batch = nleaves;
      gemm_df<float2, double, double>(g, scratch, st);
    }
  }
  // Woodbury correction of level l on q columns (in place): within each node v of level l,
  // out_v <- out_v - U_v C_v^{-1} P_v out_v with the stored U = K~_child^{-1} [W; X] and
  // CP = C^{-1} P, processed in column chunks that fit the coefficient buffers.
  void woodbury64(int l, double* out, long long ldo, int q) {
    int wl = w[l];
    if (wl == 0 || q == 0) return;
    int m = msize(l), np = npairs(l), nbk = 1 << l;
    for (int c0 = 0; c0 < q; c0 += q64max) {
      const int qq = std::min(q64max, q - c0);
      double* o = out + (size_t)c0 * ldo;
      GemmArgs g;
      g.M = qq; g.N = wl; g.K = m;
      g.A = o; g.lda = ldo; g.sA = m; g.tA = 1;
      g.B = F[l]; g.ldb = N; g.sB = m;
      g.C = fg64; g.ldc = qq; g.sC = (long long)qq * wl; g.batch = nbk;
      g64<double, T>(g);
      GemmArgs h;
      h.M = qq; h.N = 2 * wl; h.K = 2 * wl;
      h.A = fg64; h.lda = qq; h.sA = 2LL * qq * wl;
      h.B = CP64[l]; h.ldb = 2 * wl; h.sB = 4LL * wl * wl; h.tB = 1;
      h.C = stb64; h.ldc = qq; h.sC = 2LL * qq * wl; h.batch = np;
      g64<double, double>(h);
      GemmArgs k;
      k.M = m; k.N = qq; k.K = wl;
      k.A = U[l]; k.lda = N; k.sA = m;
      k.B = stb64; k.ldb = qq; k.sB = (long long)qq * wl; k.tB = 1;
      k.C = o; k.ldc = ldo; k.sC = m;
      k.alpha = -1.0; k.beta = 1.0; k.batch = nbk;
      g64<double, double>(k);
    }
  }

  // Factorization (App. C), finest level first.  The panels U_l = K~_child^{-1} [W; X] of all
  // levels sit side by side (coarse to fine) in one buffer: every panel first gets its leaf
  // solve, and once level l is factored its Woodbury correction is applied to all coarser
  // panels at once (one wide product per level instead of one per panel and level).
  void factor() {
    double* sg = sgbuf;  // Grams of the child blocks (FP64): even -> Sw, odd -> Sx
    double* Fd = (double*)WZ;   // FP64 copy of a factor panel (N x wl)
    std::vector<long long> off(tau + 2, 0);
    for (int l = 1; l <= tau; ++l) {
      off[l + 1] = off[l] + w[l];
      U[l] = Ucat + (size_t)N * off[l];
    }
    for (int l = 1; l <= tau; ++l) {
      if (w[l] == 0) continue;
      convert<T, double>(F[l], Fd, (long long)N * w[l], st);
      leaf_solve64(Fd, N, U[l], N, w[l]);
    }
    for (int l = tau; l >= 1; --l) {
      int wl = w[l];
      int np = npairs(l);
      if (wl == 0) {
        fill<double>(d_nodelog[l], 0.0, np, st);
        continue;
      }
      // U[l] now holds [W~; X~] = K~_child^{-1} [W; X] (all finer corrections applied)
      {
        GemmArgs g;
        int m = msize(l);
        g.M = wl; g.N = wl; g.K = m;
        g.A = F[l]; g.lda = N; g.sA = m; g.tA = 1;
        g.B = U[l]; g.ldb = N; g.sB = m;
        g.C = sg; g.ldc = wl; g.sC = (long long)wl * wl; g.batch = 1 << l;
        FP64Only exact;
        g64<T, double>(g);
      }
      const long long w2 = (long long)wl * wl;
      // split into Sw (even blocks) and Sx (odd blocks)
      copy_blocks<double, double>(np, wl, wl, sg, wl, 2 * w2, sw, wl, w2, 1.0, st);
      copy_blocks<double, double>(np, wl, wl, sg + w2, wl, 2 * w2, sx, wl, w2, 1.0, st);
      HODLR_CUDA(cudaMemcpyAsync(lw, sw, sizeof(double) * np * w2, cudaMemcpyDeviceToDevice, st));
      potrf_lower(np, wl, lw, wl, w2, d_rank[l], nullptr, d_status, st);     // Sw (+I padded) = Lw Lw^T
      // use the padded Sw consistently: Sw <- Lw Lw^T
      dgemm_small(np, wl, lw, 0, lw, 1, sw, 1.0, 0.0);
      dgemm_small(np, wl, sx, 0, lw, 0, t1, 1.0, 0.0);                        // Sx Lw
      dgemm_small(np, wl, lw, 1, t1, 0, t2, -1.0, 0.0);                       // -Lw^T Sx Lw
      shift_identity(np, wl, t2, wl, w2, 1.0, 1.0, st);                       // E = I - Lw^T Sx Lw
      potrf_lower(np, wl, t2, wl, w2, nullptr, d_nodelog[l], d_status, st);  // E = LE LE^T
      trtri_lower(np, wl, t2, wl, w2, t3, st);                                // LE^{-1}
      dgemm_small(np, wl, lw, 0, t3, 1, t1, 1.0, 0.0);                        // V = Lw LE^{-T}
      dgemm_small(np, wl, t1, 0, t1, 1, t2, 1.0, 0.0);                        // Lw E^{-1} Lw^T
      dgemm_small(np, wl, sx, 0, t2, 0, phi, 1.0, 0.0);                       // Sx Lw E^{-1} Lw^T
      shift_identity(np, wl, phi, wl, w2, 1.0, 1.0, st);                      // Phi = (I - Sx Sw)^{-1}
      dgemm_small(np, wl, phi, 0, sx, 0, t1, 1.0, 0.0);                       // Phi Sx
      dgemm_small(np, wl, sw, 0, phi, 0, t2, 1.0, 0.0);                       // Sw Phi
      dgemm_small(np, wl, sw, 0, t1, 0, t3, 1.0, 0.0);                        // Sw Phi Sx
      shift_identity(np, wl, t3, wl, w2, 1.0, 1.0, st);                       // I + Sw Phi Sx
      // CP = C^{-1} P = [[-Phi Sx, Phi], [I + Sw Phi Sx, -Sw Phi]]  (2wl x 2wl)
      const long long s4 = 4 * w2, ld2 = 2 * wl;
      double* cp = CP64[l];
      copy_blocks<double, double>(np, wl, wl, t1, wl, w2, cp, ld2, s4, -1.0, st);
      copy_blocks<double, double>(np, wl, wl, phi, wl, w2, cp + wl * ld2, ld2, s4, 1.0, st);
      copy_blocks<double, double>(np, wl, wl, t3, wl, w2, cp + wl, ld2, s4, 1.0, st);
      copy_blocks<double, double>(np, wl, wl, t2, wl, w2, cp + wl + wl * ld2, ld2, s4, -1.0, st);
      convert<double, T>(cp, CP[l], (long long)np * s4, st);
      status_check("SMW core");
      woodbury64(l, Ucat, N, (int)off[l]);                                  // coarser panels
    }
    // total log-det: leaves + nodes (Sylvester)
    sum_doubles(leaflog, nleaves, res + 0, 0, st);
    for (int l = 1; l <= tau; ++l) sum_doubles(d_nodelog[l], npairs(l), res + 0, 1, st);
    if (graph_mode) return;   // res[0] is read on the device
    HODLR_CUDA(cudaMemcpyAsync(&logdet, res, sizeof(double), cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
    if (!std::isfinite(logdet)) throw Error(HODLR_ENUMERIC, "log-determinant is not finite");
  }
  void dgemm_small(int nb, int n, const double* a, int ta, const double* b, int tb, double* cc, double alpha,
                   double beta) {
    GemmArgs g;
    g.M = n; g.N = n; g.K = n;
    g.A = a; g.lda = n; g.sA = (long long)n * n; g.tA = ta;
    g.B = b; g.ldb = n; g.sB = (long long)n * n; g.tB = tb;
    g.C = cc; g.ldc = n; g.sC = (long long)n * n;
    g.alpha = alpha; g.beta = beta; g.batch = nb;
    g64<double, double>(g);
  }

  // ---------------------------------------------------------------- HODLR products (mixed vector type V)
  // out = M X for M = K~ (j<0) or K~_j, at depth d: leaves + off-diagonal levels > d
  template <class V>
  void matvec(int j, const V* X, long long ldx, V* out, long long ldo, int q, int d) {
    const int nl = leaf;
    const T* Lf = j < 0 ? A : dA[j];
    {
      GemmArgs g;
      g.M = nl; g.N = q; g.K = nl;
      g.A = Lf; g.lda = nl; g.sA = (long long)nl * nl;
      g.B = X; g.ldb = ldx; g.sB = nl;
      g.C = out; g.ldc = ldo; g.sC = nl; g.batch = nleaves;
      gemm<T, V, V, V>(g, scratch, st);
    }
    for (int l = d + 1; l <= tau; ++l) {
      int wl = w[l];
      if (wl == 0) continue;
      int m = msize(l), nbk = 1 << l;
      const int wl4 = (wl + 3) & ~3;
      V* tp = (V*)tpan;
      auto tn = [&](const T* Fp, V* C) {
        GemmArgs g;
        g.M = wl; g.N = q; g.K = m;
        g.A = Fp; g.lda = N; g.sA = m; g.tA = 1;
        g.B = X; g.ldb = ldx; g.sB = m;
        g.C = C; g.ldc = wl4; g.sC = (long long)wl4 * q; g.batch = nbk;
        gemm<T, V, V, V>(g, scratch, st);
      };
      auto nn = [&](const T* Fp, const V* Bp) {
        GemmArgs g;
        g.M = m; g.N = q; g.K = wl;
        g.A = Fp; g.lda = N; g.sA = m;
        g.B = Bp; g.ldb = wl4; g.sB = (long long)wl4 * q; g.bmap = BMAP_XOR1;
        g.C = out; g.ldc = ldo; g.sC = m;
        g.beta = 1.0; g.batch = nbk;
        gemm<T, V, V, V>(g, scratch, st);
      };
      if (j < 0) {
        tn(F[l], tp);
        nn(F[l], tp);
      } else {
        V* tp2 = tp + (size_t)nbk * wl4 * q;
        tn(F[l], tp);
        tn(dF[j][l], tp2);
        nn(dF[j][l], tp);
        nn(F[l], tp2);
      }
    }
  }

  // ---------------------------------------------------------------- K~^{-1} b
  // alpha = K~^{-1} b for a tree-order FP64 vector: FP64 solve against the stored K~ (its
  // factors are exact in the stored precision, so no refinement is needed).
  void solve_tree(const double* b, double* x) { solve64(b, N, x, N, 1, 0); }

  // ---------------------------------------------------------------- exact traces (App. B)
  // t[i] = tr(K~^{-1} M_i), f[i][j] = tr(K~^{-1} M_i K~^{-1} M_j), M = (I, K~_ell, K~_kappa)
  void traces_impl(bool fisher, double* t_out, double* f_out) {
    const int nl = leaf;
    double* acc = res + 16;   // 3 + 9 accumulators
    HODLR_CUDA(cudaMemsetAsync(acc, 0, 12 * sizeof(double), st));
    // leaves: Lambda_0 = A^{-1}, Lambda_i = A^{-1} dA_i
    T* Lam = WZ;
    const long long nl2 = (long long)nl * nl;
    HODLR_CUDA(cudaMemcpyAsync(Lam, Ainv, sizeof(T) * nleaves * nl2, cudaMemcpyDeviceToDevice, st));
    for (int i = 0; i < 2; ++i) {
      GemmArgs g;
      g.M = nl; g.N = nl; g.K = nl;
      g.A = Ainv; g.lda = nl; g.sA = nl2;
      g.B = dA[i]; g.ldb = nl; g.sB = nl2;
      g.C = Lam + (size_t)(i + 1) * nleaves * nl2; g.ldc = nl; g.sC = nl2; g.batch = nleaves;
      gemmT(g);
    }
    for (int i = 0; i < 3; ++i) {
      const T* Li = Lam + (size_t)i * nleaves * nl2;
      trace_products<T>(nleaves, nl, nullptr, Li, nl, nl2, nullptr, 0, 0, 0, red, st);
      sum_doubles(red, nleaves, acc + i, 1, st);
      if (!fisher) continue;
      for (int j = i; j < 3; ++j) {
        const T* Lj = Lam + (size_t)j * nleaves * nl2;
        trace_products<T>(nleaves, nl, nullptr, Li, nl, nl2, Lj, nl, nl2, 0, red, st);
        sum_doubles(red, nleaves, acc + 3 + 3 * i + j, 1, st);
      }
    }
    // nodes, level by level
    for (int l = 1; l <= tau; ++l) {
      int wl = w[l];
      if (wl == 0) continue;
      const int np = npairs(l), m = msize(l), w2 = 2 * wl;
      const long long pw = (long long)N * w2;   // one 2wl-wide panel
      // WP = [P | Y1 | Y2 | Pi1 | Pi2]; P = U_v as a panel: c1 rows [W~, 0], c2 rows [0, X~]
      T* P = WP;
      fill<T>(P, T(0), pw, st);
      copy_blocks<double, T>(np, m, wl, U[l], N, 2LL * m, P, N, 2LL * m, 1.0, st);
      copy_blocks<double, T>(np, m, wl, U[l] + m, N, 2LL * m, P + m + (size_t)wl * N, N, 2LL * m, 1.0, st);
      for (int i = 0; i < 2; ++i) matvec<T>(i, P, N, P + (size_t)(i + 1) * pw, N, w2, l - 1);
      int nsolve = 3;
      if (fisher) {
        for (int i = 0; i < 2; ++i) {
          // Pi_i: c1 rows [dQ | Q], c2 rows [B~ | dB~]
          T* Pi = P + (size_t)(3 + i) * pw;
          copy_blocks<T, T>(np, m, wl, dF[i][l], N, 2LL * m, Pi, N, 2LL * m, 1.0, st);
          copy_blocks<T, T>(np, m, wl, F[l], N, 2LL * m, Pi + (size_t)wl * N, N, 2LL * m, 1.0, st);
          copy_blocks<T, T>(np, m, wl, F[l] + m, N, 2LL * m, Pi + m, N, 2LL * m, 1.0, st);
          copy_blocks<T, T>(np, m, wl, dF[i][l] + m, N, 2LL * m, Pi + m + (size_t)wl * N, N, 2LL * m, 1.0, st);
        }
        nsolve = 5;
        solve_depth(P, N, WZ, N, nsolve * w2, l);
      }
      // per-node Grams (2wl x 2wl): G_i = P^T Y_i
      const long long g2 = (long long)w2 * w2;
      T* Gm = nodeG;               // 3 blocks of np * g2
      T* Tm = nodeG + 3 * np * g2; // 6 blocks
      T* Xm = nodeX;               // CP G_i
      for (int i = 0; i < 3; ++i) node_tn(l, w2, P, P + (size_t)i * pw, Gm + (size_t)i * np * g2);
      for (int i = 0; i < 3; ++i) dgemm_nodes(np, w2, CP[l], Gm + (size_t)i * np * g2, Xm + (size_t)i * np * g2);
      for (int i = 0; i < 3; ++i) {
        trace_products<T>(np, w2, nullptr, Xm + (size_t)i * np * g2, w2, g2, nullptr, 0, 0, 0, red, st);
        sum_doubles_scaled(red, np, acc + i, -1.0);
      }
      if (!fisher) continue;
      int tix = 0;
      for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j, ++tix) {
          T* Tij = Tm + (size_t)tix * np * g2;
          node_tn(l, w2, P + (size_t)i * pw, WZ + (size_t)j * pw, Tij);       // T_ij = Y_i^T Z_j
          // - tr(CP T_ij) - tr(CP T_ij^T)
          trace_products<T>(np, w2, nullptr, CP[l], w2, g2, Tij, w2, g2, 0, red, st);
          sum_doubles_scaled(red, np, acc + 3 + 3 * i + j, -1.0);
          trace_products<T>(np, w2, nullptr, CP[l], w2, g2, Tij, w2, g2, 1, red, st);
          sum_doubles_scaled(red, np, acc + 3 + 3 * i + j, -1.0);
          // + tr((CP G_i)(CP G_j))
          trace_products<T>(np, w2, nullptr, Xm + (size_t)i * np * g2, w2, g2, Xm + (size_t)j * np * g2, w2, g2, 0,
                            red, st);
          sum_doubles_scaled(red, np, acc + 3 + 3 * i + j, 1.0);
          // cross term of the two off-diagonal blocks: 2 tr((A_j^T K1^{-1} A_i)(B_i^T K2^{-1} B_j))
          if (i >= 1 && j >= 1) {
            T* Pi_i = P + (size_t)(2 + i) * pw;
            T* Pi_j = P + (size_t)(2 + j) * pw;
            T* Pb_i = WZ + (size_t)(2 + i) * pw;
            T* Pb_j = WZ + (size_t)(2 + j) * pw;
            T* Gji = nodeX + 3 * np * g2;       // per child block (2^l blocks)
            T* Gij = Gji + (size_t)2 * np * g2;
            child_tn(l, w2, Pi_j, Pb_i, Gji);   // Gamma_ji[b] = Pi_j[b]^T Pibar_i[b]
            child_tn(l, w2, Pi_i, Pb_j, Gij);   // Gamma_ij[b]
            // tr(Gamma_ji[c1] Gamma_ij[c2]): even blocks of Gji with odd blocks of Gij
            trace_products<T>(np, w2, nullptr, Gji, w2, 2 * g2, Gij + g2, w2, 2 * g2, 0, red, st);
            sum_doubles_scaled(red, np, acc + 3 + 3 * i + j, 2.0);
          }
        }
    }
    if (graph_mode) return;   // the accumulators are read on the device
    double h[12];
    HODLR_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < 3; ++i) t_out[i] = h[i];
    if (fisher)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) f_out[3 * i + j] = i <= j ? h[3 + 3 * i + j] : h[3 + 3 * j + i];
  }
  // per-node (rows of both children) Gram C_v = A_v^T B_v, 2w x 2w
  void node_tn(int l, int w2, const T* Ap, const T* Bp, T* Cp) {
    int mm = 2 * msize(l);
    GemmArgs g;
    g.M = w2; g.N = w2; g.K = mm;
    g.A = Ap; g.lda = N; g.sA = mm; g.tA = 1;
    g.B = Bp; g.ldb = N; g.sB = mm;
    g.C = Cp; g.ldc = w2; g.sC = (long long)w2 * w2; g.batch = npairs(l);
    gemmT(g);
  }
  void child_tn(int l, int w2, const T* Ap, const T* Bp, T* Cp) {
    int mm = msize(l);
    GemmArgs g;
    g.M = w2; g.N = w2; g.K = mm;
    g.A = Ap; g.lda = N; g.sA = mm; g.tA = 1;
    g.B = Bp; g.ldb = N; g.sB = mm;
    g.C = Cp; g.ldc = w2; g.sC = (long long)w2 * w2; g.batch = 1 << l;
    gemmT(g);
  }
  void dgemm_nodes(int np, int w2, const T* a, const T* b, T* cc) {
    GemmArgs g;
    g.M = w2; g.N = w2; g.K = w2;
    g.A = a; g.lda = w2; g.sA = (long long)w2 * w2;
    g.B = b; g.ldb = w2; g.sB = (long long)w2 * w2;
    g.C = cc; g.ldc = w2; g.sC = (long long)w2 * w2; g.batch = np;
    gemmT(g);
  }
  void sum_doubles_scaled(double* x, int n, double* out, double scale);

  void traces(double* t, double* f) override {
    if (!built) throw Error(HODLR_EINVAL, "no build");
    derivatives_supported();
    traces_impl(true, t, f);
    t[0] -= npad;   // padding rows: a unit diagonal, decoupled (see eval)
    f[0] -= npad;
  }
  // The FP32 sketch of the mixed path carries rounding of relative size 6e-8 into dY, which
  // Alg. 2 multiplies by cond(R) (up to 1/guard = 1e5) in dY R^{-1}; with the bivariate
  // model's leaf conditioning (~1e6) the resulting score and Fisher entries are not
  // accurate, so they are refused there (the likelihood itself is unaffected).
  void derivatives_supported() const {
    if (sizeof(T) == 4 && nvar == 2)
      throw Error(HODLR_ENOTIMPL, "score and Fisher of bivariate models need the FP64 path");
  }

  // ---------------------------------------------------------------- likelihood, gradient, Fisher
  void eval(const double* theta, const double* y, double* nll, double* grad, double* fisher) override {
    if (grad || fisher) derivatives_supported();
    bool same = built;
    for (int k = 0; k < 4; ++k) same = same && theta[k] == theta_built[k];
    if (!same) build(theta);
    const double s2 = theta[0], t2 = theta[3];
    double a_y = 0.0, a_a = 0.0, aKa[2] = {0, 0};
    if (nll || grad) {
      if (!y) throw Error(HODLR_EINVAL, "y is required");
      HODLR_CUDA(cudaMemsetAsync(d_status + 1, 0, sizeof(int), st));
      check_finite<double>(y, Nr, d_status + 1, st);
      permute_rows<double, double>(y, Nr, vec_d, N, d_perm_plain, N, 1, 0, st);   // y in tree order
      solve_tree(vec_d, vec_d + N);                                               // alpha
      double* alpha = vec_d + N;
      dot_columns<double, double>(N, 1, vec_d, N, alpha, N, res + 40, st);        // y^T alpha
      dot_columns<double, double>(N, 1, alpha, N, alpha, N, res + 41, st);        // alpha^T alpha
      if (grad) {
        for (int j = 0; j < 2; ++j) {
          matvec<double>(j, alpha, N, vec_d2, N, 1, 0);
          dot_columns<double, double>(N, 1, alpha, N, vec_d2, N, res + 42 + j, st);
        }
      }
      double h[4];
      int bad = 0;
      HODLR_CUDA(cudaMemcpyAsync(h, res + 40, sizeof(h), cudaMemcpyDeviceToHost, st));
      HODLR_CUDA(cudaMemcpyAsync(&bad, d_status + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      HODLR_CUDA(cudaStreamSynchronize(st));
      if (bad) throw Error(HODLR_ENUMERIC, "y has NaN or Inf");
      a_y = h[0]; a_a = h[1]; aKa[0] = h[2]; aKa[1] = h[3];
    }
    double t[3] = {0, 0, 0}, f[9] = {0};
    if (grad || fisher) {
      traces_impl(fisher != nullptr, t, f);
      // padding rows carry a unit diagonal decoupled from everything else: they add 1 each to
      // tr(K~^{-1}) and tr(K~^{-2}) and nothing to any other trace
      t[0] -= npad;
      f[0] -= npad;
    }
    const double n = (double)Nr;
    double out_nll = 0.5 * n * log(2.0 * M_PI) + 0.5 * logdet + 0.5 * a_y;
    // traces of K~^{-1} K~_j: sigma2 -> (N - tau2 t0)/sigma2, ell -> t1, kappa -> t2, tau2 -> t0
    double trj[4] = {(n - t2 * t[0]) / s2, t[1], t[2], t[0]};
    double quad[4] = {(a_y - t2 * a_a) / s2, aKa[0], aKa[1], a_a};
    if (nll) *nll = out_nll;
    if (grad)
      for (int j = 0; j < 4; ++j) grad[j] = 0.5 * trj[j] - 0.5 * quad[j];
    if (fisher) {
      // F_ab = tr(K~^{-1} M_a K~^{-1} M_b) for M in (I, K_ell, K_kappa): f[3a+b]
      // K~_sigma2 = (K~ - tau2 I)/sigma2:
      //   tr(K^-1 Ks K^-1 M) = (t_M - tau2 f_{0M})/sigma2,  tr(K^-1 Ks K^-1 Ks) = (N - 2 tau2 t0 + tau2^2 f00)/sigma2^2
      auto F3 = [&](int a, int b) { return f[3 * a + b]; };
      double I4[4][4];
      int map[4] = {-1, 1, 2, 0};   // parameter -> index in (I, ell, kappa); -1 = sigma2
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          int ia = map[a], ib = map[b];
          double v;
          if (ia < 0 && ib < 0) v = (n - 2.0 * t2 * t[0] + t2 * t2 * F3(0, 0)) / (s2 * s2);
          else if (ia < 0) v = (t[ib] - t2 * F3(0, ib)) / s2;
          else if (ib < 0) v = (t[ia] - t2 * F3(0, ia)) / s2;
          else v = F3(ia, ib);
          I4[a][b] = 0.5 * v;
        }
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) fisher[4 * a + b] = I4[a][b];
    }
    bool fin = std::isfinite(out_nll);
    if (grad) for (int j = 0; j < 4; ++j) fin = fin && std::isfinite(grad[j]);
    if (fisher) for (int j = 0; j < 16; ++j) fin = fin && std::isfinite(fisher[j]);
    if (!fin) throw Error(HODLR_ENUMERIC, "non-finite result");
  }

  // NLL and gradient without host synchronisation (for capture into a CUDA graph); the same
  // arithmetic as eval(), with the scalar assembly done by finalize_nll_grad on the device.
  void eval_graph(const double* theta, const double* y) override {
    if (!graph_mode) throw Error(HODLR_EINVAL, "eval_graph outside graph mode");
    derivatives_supported();
    build(theta);
    HODLR_CUDA(cudaMemsetAsync(d_status + 1, 0, sizeof(int), st));
    check_finite<double>(y, Nr, d_status + 1, st);
    permute_rows<double, double>(y, Nr, vec_d, N, d_perm_plain, N, 1, 0, st);
    solve_tree(vec_d, vec_d + N);
    double* alpha = vec_d + N;
    dot_columns<double, double>(N, 1, vec_d, N, alpha, N, res + 40, st);
    dot_columns<double, double>(N, 1, alpha, N, alpha, N, res + 41, st);
    for (int j = 0; j < 2; ++j) {
      matvec<double>(j, alpha, N, vec_d2, N, 1, 0);
      dot_columns<double, double>(N, 1, alpha, N, vec_d2, N, res + 42 + j, st);
    }
    traces_impl(false, nullptr, nullptr);
    finalize_nll_grad(theta);
  }
  const double* graph_out() const override { return res + 200; }
  void finalize_nll_grad(const double* theta);

  // ---------------------------------------------------------------- test entry points
  void apply_nat(const double* theta, int which, const double* X, double* Yo, int ncols) override {
    for (int k = 0; k < 4; ++k) theta_built[k] = theta[k];
    built = false;
    set_physics(theta);
    // natural -> tree (T), apply, tree -> natural (double)
    for (int c0 = 0; c0 < ncols; c0 += c) {
      int qq = std::min(c, ncols - c0);
      permute_rows<double, T>(X + (size_t)c0 * Nr, Nr, R, N, d_perm_plain, N, qq, 0, st);
      T* o = KR;
      if (which == 0) apply(R, N, qq, o, nullptr, nullptr, N);
      else if (which == 2) apply(R, N, qq, nullptr, o, nullptr, N);
      else if (which == 3) apply(R, N, qq, nullptr, nullptr, o, N);
      else if (which == 1) {
        apply(R, N, qq, o, nullptr, nullptr, N);
        axpby<T>(N, qq, -theta[3] / theta[0], R, N, 1.0 / theta[0], o, N, st);
      } else if (which == 4) {
        HODLR_CUDA(cudaMemcpyAsync(o, R, sizeof(T) * (size_t)N * qq, cudaMemcpyDeviceToDevice, st));
      } else throw Error(HODLR_EINVAL, "which");
      permute_rows<T, double>(o, N, Yo + (size_t)c0 * Nr, Nr, d_perm_plain, N, qq, 1, st);
    }
    if (tc_status_take(st)) throw Error(HODLR_ETIMEOUT, "a tensor-core product gave up waiting for its operands");
  }
  void probe(int level, int ncols, double* out) override {
    if (level < 1 || level > tau || ncols > c) throw Error(HODLR_EINVAL, "level / ncols");
    probe_panel<T>(N, ncols, level, 0, seed, d_mask[level], d_rowid, R, N, st);
    permute_rows<T, double>(R, N, out, Nr, d_real2pad, Nr, ncols, 0, st);   // real tree rows
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  void densify(int which, double* out) override {
    if (!built) throw Error(HODLR_EINVAL, "no build");
    if ((long long)N * N > (1LL << 28)) throw Error(HODLR_EINVAL, "densify is for small N only");
    // columns of the identity (at the real rows) through the HODLR product, rows compacted to
    // the real tree order
    int j = which == 0 || which == 1 || which == 4 ? -1 : which - 2;
    const int qd = (int)std::max<size_t>(1, std::min<size_t>(64, (size_t)wide * sizeof(T) / sizeof(double)));
    double* X = (double*)WZ;
    double* Yp = (double*)WP;
    for (int c0 = 0; c0 < Nr; c0 += qd) {
      int qq = std::min(qd, Nr - c0);
      fill<double>(X, 0.0, (long long)N * qq, st);
      set_unit(X, c0, qq);
      matvec<double>(j, (const double*)X, N, Yp, N, qq, 0);
      if (which == 1) axpby<double>(N, qq, -theta_built[3] / theta_built[0], (const double*)X, N,
                                    1.0 / theta_built[0], Yp, N, st);
      if (which == 4) HODLR_CUDA(cudaMemcpyAsync(Yp, X, sizeof(double) * (size_t)N * qq, cudaMemcpyDeviceToDevice, st));
      permute_rows<double, double>(Yp, N, out + (size_t)c0 * Nr, Nr, d_real2pad, Nr, qq, 0, st);
    }
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  void set_unit(double* col, int c0, int qq);
  void grad_adjoint(const double* y, double* g) override;
  void debug_level(int what, int level, double* out, int64_t count, int32_t* w_out) override {
    if (!built || level < 1 || level > tau) throw Error(HODLR_EINVAL, "level");
    int wl = w[level];
    *w_out = wl;
    size_t n = (what <= 1) ? (size_t)Nr * wl : (size_t)npairs(level) * wl * wl;
    if ((int64_t)n > count) throw Error(HODLR_EINVAL, "count");
    double* tmp = vec_d2;
    if (what <= 1) {
      // panels in the real tree order (padding rows dropped)
      if (what == 0) permute_rows<T, double>(F[level], N, (double*)WZ, Nr, d_real2pad, Nr, wl, 0, st);
      else permute_rows<double, double>(U[level], N, (double*)WZ, Nr, d_real2pad, Nr, wl, 0, st);
      HODLR_CUDA(cudaMemcpyAsync(out, WZ, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    } else {
      // recompute the child Grams of this level from F and U (as factor() does)
      GemmArgs g;
      int m = msize(level);
      g.M = wl; g.N = wl; g.K = m;
      g.A = F[level]; g.lda = N; g.sA = m; g.tA = 1;
      g.B = U[level]; g.ldb = N; g.sB = m;
      g.C = sgbuf; g.ldc = wl; g.sC = (long long)wl * wl; g.batch = 1 << level;
      g64<T, double>(g);
      const long long w2 = (long long)wl * wl;
      copy_blocks<double, double>(npairs(level), wl, wl, sgbuf + (what == 3 ? w2 : 0), wl, 2 * w2, sw, wl, w2, 1.0, st);
      HODLR_CUDA(cudaMemcpyAsync(out, sw, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    (void)tmp;
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  void logdet_levels(double* out) override {
    if (!built) throw Error(HODLR_EINVAL, "no build");
    sum_doubles(leaflog, nleaves, res + 60, 0, st);
    for (int l = 1; l <= tau; ++l) sum_doubles(d_nodelog[l], npairs(l), res + 60 + l, 0, st);
    HODLR_CUDA(cudaMemcpyAsync(out, res + 60, sizeof(double) * (tau + 1), cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  // Y = K~ X (which 0) or K~_j X (which 1..4: sigma2, ell, kappa, tau2), natural order
  void matvec_nat(int which, const double* X, double* Y, int ncols) override {
    if (!built) throw Error(HODLR_EINVAL, "no build");
    const int j = which == 0 || which == 1 || which == 4 ? -1 : which - 2;
    const int qd = (int)std::max<size_t>(1, std::min<size_t>(64, (size_t)wide * sizeof(T) / sizeof(double)));
    double* Xp = (double*)WZ;
    double* Yp = (double*)WP;
    for (int c0 = 0; c0 < ncols; c0 += qd) {
      const int qq = std::min(qd, ncols - c0);
      permute_rows<double, double>(X + (size_t)c0 * Nr, Nr, Xp, N, d_perm_plain, N, qq, 0, st);   // padding rows 0
      if (which == 4) {
        HODLR_CUDA(cudaMemcpyAsync(Yp, Xp, sizeof(double) * (size_t)N * qq, cudaMemcpyDeviceToDevice, st));
      } else {
        matvec<double>(j, (const double*)Xp, N, Yp, N, qq, 0);
        // K~_sigma2 = (K~ - tau2 I) / sigma2
        if (which == 1) axpby<double>(N, qq, -theta_built[3] / theta_built[0], (const double*)Xp, N,
                                      1.0 / theta_built[0], Yp, N, st);
      }
      permute_rows<double, double>(Yp, N, Y + (size_t)c0 * Nr, Nr, d_perm_plain, N, qq, 1, st);
    }
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  void solve_nat(const double* b, double* x) override {
    if (!built) throw Error(HODLR_EINVAL, "no build");
    permute_rows<double, double>(b, Nr, vec_d, N, d_perm_plain, N, 1, 0, st);
    solve_tree(vec_d, vec_d + N);
    permute_rows<double, double>(vec_d + N, N, x, Nr, d_perm_plain, N, 1, 1, st);
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
  void set_pivots(const int32_t* piv) override {
    if (!piv) { frozen = false; return; }
    size_t off = 0;
    for (int l = 1; l <= tau; ++l) {
      HODLR_CUDA(cudaMemcpyAsync(d_piv[l], piv + off, sizeof(int) * (size_t)npairs(l) * c, cudaMemcpyHostToDevice, st));
      off += (size_t)npairs(l) * c;
    }
    HODLR_CUDA(cudaStreamSynchronize(st));
    frozen = true;
    built = false;
  }
  void read_perm(int64_t* perm) override {
    std::vector<int> pp(N), rid(d_rowid ? N : 0);
    HODLR_CUDA(cudaMemcpyAsync(pp.data(), d_perm_plain, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, st));
    if (d_rowid) HODLR_CUDA(cudaMemcpyAsync(rid.data(), d_rowid, sizeof(int) * (size_t)N, cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
    for (int i = 0; i < N; ++i) {
      const int pos = d_rowid ? rid[i] : i;
      if (pos >= 0) perm[pos] = pp[i];
    }
  }
  void get_pivots(int32_t* piv) const override {
    size_t off = 0;
    for (int l = 1; l <= tau; ++l) {
      HODLR_CUDA(cudaMemcpy(piv + off, d_piv[l], sizeof(int) * (size_t)npairs(l) * c, cudaMemcpyDeviceToHost));
      off += (size_t)npairs(l) * c;
    }
  }
};

// small kernels local to the engine
namespace {
template <class T>
__global__ void identity_blocks_kernel(const int* counts, int nl, T* S, long long ld) {
  int b = blockIdx.x;
  int lo = b * nl, n = counts[b];   // leaf slot b: its real rows first, then padding rows
  for (int i = threadIdx.x; i < n; i += blockDim.x) S[lo + i + (size_t)i * ld] = T(1);
}
// rows [p*stride, p*stride + m) of pair p: columns j >= rank[p] set to zero
template <class T>
__global__ void zero_pad_cols_kernel(int m, long long stride, int wl, const int* rank, T* rows, long long ld) {
  int p = blockIdx.y;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * wl) return;
  int i = (int)(e % m), j = (int)(e / m);
  if (j >= rank[p]) rows[p * stride + i + (size_t)j * ld] = T(0);
}
__global__ void identity_cols_kernel(const int* counts, int nl, double* S, long long ld, int j0, int qq) {
  int b = blockIdx.x;
  int lo = b * nl, n = counts[b];
  for (int jj = threadIdx.x; jj < qq; jj += blockDim.x)
    if (j0 + jj < n) S[lo + j0 + jj + (size_t)jj * ld] = 1.0;
}
template <class TS, class TD>
__global__ void scatter_leaf_cols_kernel(const int* counts, int nl, const TS* E, long long lde, int j0, int qq,
                                         TD* Ablk) {
  int b = blockIdx.y;
  int lo = b * nl, n = counts[b];
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nl * qq) return;
  int i = (int)(e % nl), jj = (int)(e / nl);
  int j = j0 + jj;
  double v = 0.0;
  if (i < n && j < n) v = (double)E[lo + i + (size_t)jj * lde];
  else if (i == j) v = 1.0;
  Ablk[(size_t)b * nl * nl + i + (size_t)j * nl] = (TD)v;
}
template <class V>
__global__ void symmetrize_blocks_kernel(int nl, V* Ablk) {
  int b = blockIdx.y;
  V* Ab = Ablk + (size_t)b * nl * nl;
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)nl * nl) return;
  int i = (int)(e % nl), j = (int)(e / nl);
  if (i <= j) return;
  V a = Ab[i + (size_t)j * nl], c = Ab[j + (size_t)i * nl];
  V v = (V)(0.5 * ((double)a + (double)c));
  Ab[i + (size_t)j * nl] = v;
  Ab[j + (size_t)i * nl] = v;
}
// column j of X (ld N) = the unit vector of real tree position c0 + j
__global__ void unit_cols_kernel(double* col, long long N, const int* real2pad, int c0, int qq) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < qq) col[real2pad[c0 + j] + (size_t)j * N] = 1.0;
}
__global__ void scale_sum_kernel(const double* x, int n, double* out, double scale) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    *out += scale * t;
  }
}
}  // namespace

// {nll, g_sigma2, g_ell, g_kappa, g_tau2, status} from the device accumulators of one evaluation
// (the formulas of eval(): log-det res[0], y^T a res[40], a^T a res[41], a^T K~_j a res[42..43],
// tr(K~^{-1} M) res[16..18] for M = (I, K~_ell, K~_kappa)).
__global__ void finalize_nll_grad_kernel(const double* res, const int* status, double nr, double npad, double s2,
                                         double t2, double* out) {
  if (threadIdx.x != 0) return;
  const double ldet = res[0], a_y = res[40], a_a = res[41];
  const double t0 = res[16] - npad;
  const double trj[4] = {(nr - t2 * t0) / s2, res[17], res[18], t0};
  const double quad[4] = {(a_y - t2 * a_a) / s2, res[42], res[43], a_a};
  const double nll = 0.5 * nr * log(2.0 * M_PI) + 0.5 * ldet + 0.5 * a_y;
  out[0] = nll;
  bool fin = isfinite(nll);
  for (int j = 0; j < 4; ++j) {
    out[1 + j] = 0.5 * trj[j] - 0.5 * quad[j];
    fin = fin && isfinite(out[1 + j]);
  }
  double st = 0.0;
  if (status[0] != 0) st = (double)status[0];
  else if (status[1] != 0 || !fin) st = (double)HODLR_ENUMERIC;
  out[5] = st;
}
template <class T> void Engine<T>::finalize_nll_grad(const double* theta) {
  finalize_nll_grad_kernel<<<1, 32, 0, st>>>(res, d_status, (double)Nr, (double)npad, theta[0], theta[3],
                                              res + 200);
  check_launch("finalize_nll_grad");
}

template <class T> void Engine<T>::identity_blocks(T* Sl) {
  identity_blocks_kernel<T><<<nleaves, 256, 0, st>>>(d_leafreal, leaf, Sl, N);
  check_launch("identity_blocks");
}
template <class T> void Engine<T>::zero_pad_cols(int l, int wl, T* rows) {
  int m = msize(l);
  dim3 g(cdiv((long long)m * wl, 256), npairs(l));
  zero_pad_cols_kernel<T><<<g, 256, 0, st>>>(m, 2LL * m, wl, d_rank[l], rows, N);
  check_launch("zero_pad_cols");
}
template <class T> void Engine<T>::identity_cols(double* Sx, int j0, int qq) {
  identity_cols_kernel<<<nleaves, 64, 0, st>>>(d_leafreal, leaf, Sx, N, j0, qq);
  check_launch("identity_cols");
}
template <class T> template <class TS, class TD> void Engine<T>::scatter_leaf_cols(const TS* E, int j0, int qq, TD* Ablk) {
  dim3 g(cdiv((long long)leaf * qq, 256), nleaves);
  scatter_leaf_cols_kernel<TS, TD><<<g, 256, 0, st>>>(d_leafreal, leaf, E, N, j0, qq, Ablk);
  check_launch("scatter_leaf_cols");
}
template <class T> template <class V> void Engine<T>::symmetrize_blocks(V* Ablk) {
  dim3 g(cdiv((long long)leaf * leaf, 256), nleaves);
  symmetrize_blocks_kernel<V><<<g, 256, 0, st>>>(leaf, Ablk);
  check_launch("symmetrize_blocks");
}
template <class T> void Engine<T>::set_unit(double* col, int c0, int qq) {
  unit_cols_kernel<<<cdiv(qq, 64), 64, 0, st>>>(col, N, d_real2pad, c0, qq);
  check_launch("unit_cols");
}
template <class T> void Engine<T>::sum_doubles_scaled(double* x, int n, double* out, double scale) {
  scale_sum_kernel<<<1, 1024, 0, st>>>(x, n, out, scale);
  check_launch("scale_sum");
}

// ---------------------------------------------------------------- reverse mode through the factorization
// The gradient of the NLL as the adjoint of the NLL with respect to the HODLR factors contracted
// with their tangents: dNLL/dtheta_j = <Kbar, K~_j>, Kbar = (K~^{-1} - alpha alpha^T) / 2, alpha =
// K~^{-1} y.  K~_j is the block-diagonal dA_j plus, per level and sibling pair, the blocks
// dB~ Q^T + B~ dQ^T (right x left) and their transposes, so
//   <Kbar, K~_j> = sum_b <Kbar_bb, dA_j,b> + sum_l <Fbar_l, dF_j,l>,
// where, for the sibling pair (c1, c2) of level l with factors Q (rows of c1) and B~ (rows of c2),
//   <Kbar, dB~ Q^T + B~ dQ^T> x 2 = <K~^{-1}[c2,c1] Q - a2 a1^T Q, dB~> + <K~^{-1}[c1,c2] B~ - a1 a2^T B~, dQ>
// (a = alpha).  The blocks of K~^{-1} follow from the stored factorization (App. C): a node's
// inverse is D^{-1} - U CP U^T with D its children's block diagonal, U = D^{-1} blockdiag(Q, B~)
// the stored panel and CP = C^{-1} P the stored core.  Hence
//   (K~^{-1})_bb = A_b^{-1} - sum_l U_l[b] CP_l[s,s] U_l[b]^T            (leaf b, side s at level l)
//   K~^{-1}[c2,c1] = -U_l[c2] CP_l[2,1] U_l[c1]^T - sum_{l'<l} U_l'[c2] CP_l'[s,s] U_l'[c1]^T
// and every term is a contraction of small products U_l'[c]^T F_l[c], U_l'[c]^T dF_l[c] of the
// stored panels: no solves besides alpha.  sigma2 and tau2 use K~_sigma2 = (K~ - tau2 I) / sigma2
// and K~_tau2 = I, which need tr K~^{-1} (the leaf blocks).
__device__ double adj_block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  return r;   // in every thread
}
// per sibling pair v of level l: -<C A_c1, B_c2> - <C' A_c2, B_c1> for j = 0, 1 into red[2v + j],
// with A_c = U_l'[c]^T F_l[c], B_c = U_l'[c]^T dF_j,l[c] (wp x wl each, stride wp*wl per child c) and
// C, C' the cores: for l' = l the off-diagonal blocks CP_l[2,1], CP_l[1,2] of the pair; for l' < l
// the diagonal block CP_l'[s,s] of the level-l' pair holding both children (C = C')
__global__ void adj_pair_kernel(int wp, int wl, bool same, long long m, long long mp, const double* cp,
                                const double* A, const double* B0, const double* B1, double* red) {
  __shared__ double sh[32];
  const int v = blockIdx.x;
  const long long wpl = (long long)wp * wl, ld2 = 2LL * wp;
  const double* A1 = A + (2LL * v) * wpl;
  const double* A2 = A1 + wpl;
  const double *C1, *C2;   // core applied to A_c1 (paired with B_c2) and to A_c2 (with B_c1)
  if (same) {
    const double* base = cp + (long long)v * 4 * wp * wp;
    C1 = base + wp;             // CP[2,1]: rows wp.., columns 0..
    C2 = base + wp * ld2;       // CP[1,2]: rows 0.., columns wp..
  } else {
    const long long anc = (2LL * v * m) / mp;          // ancestor child block at depth l'
    const double* base = cp + (anc >> 1) * 4LL * wp * wp + (anc & 1) * (long long)wp * (2 * wp + 1);
    C1 = base;
    C2 = base;
  }
  double a0 = 0.0, a1 = 0.0;
  for (long long e = threadIdx.x; e < wpl; e += blockDim.x) {
    const int r = (int)(e % wp), c = (int)(e / wp);
    double t1 = 0.0, t2 = 0.0;
    for (int k = 0; k < wp; ++k) {
      t1 += C1[r + k * ld2] * A1[k + (long long)c * wp];
      t2 += C2[r + k * ld2] * A2[k + (long long)c * wp];
    }
    a0 += t1 * B0[(2LL * v + 1) * wpl + e] + t2 * B0[(2LL * v) * wpl + e];
    a1 += t1 * B1[(2LL * v + 1) * wpl + e] + t2 * B1[(2LL * v) * wpl + e];
  }
  a0 = adj_block_sum(a0, sh);
  a1 = adj_block_sum(a1, sh);
  if (threadIdx.x == 0) {
    red[2 * v] = -a0;
    red[2 * v + 1] = -a1;
  }
}
// per sibling pair v: -(a_c1 . b_c2 + a_c2 . b_c1) with a_c = F_l[c]^T alpha_c, b_c = dF_j,l[c]^T
// alpha_c (wl each per child c) into red[2v + j]
__global__ void adj_alpha_kernel(int wl, const double* a, const double* b0, const double* b1, double* red) {
  __shared__ double sh[32];
  const int v = blockIdx.x;
  const double* a1 = a + 2LL * v * wl;
  const double* a2 = a1 + wl;
  double s0 = 0.0, s1 = 0.0;
  for (int e = threadIdx.x; e < wl; e += blockDim.x) {
    s0 += a1[e] * b0[(2LL * v + 1) * wl + e] + a2[e] * b0[2LL * v * wl + e];
    s1 += a1[e] * b1[(2LL * v + 1) * wl + e] + a2[e] * b1[2LL * v * wl + e];
  }
  s0 = adj_block_sum(s0, sh);
  s1 = adj_block_sum(s1, sh);
  if (threadIdx.x == 0) {
    red[2 * v] = -s0;
    red[2 * v + 1] = -s1;
  }
}
// per leaf b: <A_b^{-1}, dA_j,b> (j = 0, 1) and tr A_b^{-1} over the real rows
template <class T>
__global__ void adj_leaf_inv_kernel(int leaf, const int* leafreal, const T* Ainv, const T* dA0, const T* dA1,
                                    double* red) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const long long nl2 = (long long)leaf * leaf;
  double a0 = 0.0, a1 = 0.0, tr = 0.0;
  for (int e = threadIdx.x; e < leaf * leaf; e += blockDim.x) {
    const double v = (double)Ainv[b * nl2 + e];
    a0 += v * (double)dA0[b * nl2 + e];
    a1 += v * (double)dA1[b * nl2 + e];
    const int i = e % leaf, k = e / leaf;
    if (i == k && i < leafreal[b]) tr += v;
  }
  a0 = adj_block_sum(a0, sh);
  a1 = adj_block_sum(a1, sh);
  tr = adj_block_sum(tr, sh);
  if (threadIdx.x == 0) {
    red[3 * b] = a0;
    red[3 * b + 1] = a1;
    red[3 * b + 2] = tr;
  }
}
// per leaf b: <CP_l[s, s], G_b> with G_b (w x w, stride w*w) and the core of b's level-l pair
// (2w x 2w, stride 4 w*w), s the side of the pair that b lies in (children of m rows)
__global__ void adj_cp_kernel(int leaf, int w, long long m, const double* cp, const double* G, double* red) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const long long child = (long long)b * leaf / m;
  const int side = (int)(child & 1);
  const long long pair = child >> 1;
  const double* C = cp + pair * 4LL * w * w + (long long)side * w * (2 * w + 1);
  const double* Gb = G + (long long)b * w * w;
  double a = 0.0;
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) {
    const int r = e % w, c = e / w;
    a += C[r + (long long)c * 2 * w] * Gb[e];
  }
  a = adj_block_sum(a, sh);
  if (threadIdx.x == 0) red[b] = a;
}
// per leaf b: alpha_b^T dA_j,b alpha_b (j = 0, 1)
template <class T>
__global__ void adj_leaf_quad_kernel(int leaf, const double* alpha, const T* dA0, const T* dA1, double* red) {
  __shared__ double sh[32];
  const int b = blockIdx.x;
  const long long nl2 = (long long)leaf * leaf;
  const double* ab = alpha + (size_t)b * leaf;
  double a0 = 0.0, a1 = 0.0;
  for (int e = threadIdx.x; e < leaf * leaf; e += blockDim.x) {
    const int i = e % leaf, k = e / leaf;
    const double wgt = ab[i] * ab[k];
    a0 += wgt * (double)dA0[b * nl2 + e];
    a1 += wgt * (double)dA1[b * nl2 + e];
  }
  a0 = adj_block_sum(a0, sh);
  a1 = adj_block_sum(a1, sh);
  if (threadIdx.x == 0) {
    red[2 * b] = a0;
    red[2 * b + 1] = a1;
  }
}
// out += sum_i x[i * stride], i < n (fixed order)
__global__ void adj_sum_strided_kernel(const double* x, int n, int stride, double* out) {
  __shared__ double sh[32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v += x[(size_t)i * stride];
  v = adj_block_sum(v, sh);
  if (threadIdx.x == 0) *out += v;
}
static void sum_doubles_strided_on(const double* x, int n, int stride, double* out, cudaStream_t st) {
  adj_sum_strided_kernel<<<1, 1024, 0, st>>>(x, n, stride, out);
  check_launch("adj_sum");
}
__global__ void adj_finish_kernel(const double* acc, double nr, double s2, double t2, double* g) {
  // acc: 0 <A^{-1}, dA_ell>, 1 <A^{-1}, dA_kappa>, 2 tr A^{-1} (real rows), 3 alpha^T dA_ell alpha,
  // 4 alpha^T dA_kappa alpha, 5 alpha^T y, 6 alpha^T alpha, 7 levels ell, 8 levels kappa,
  // 9..11 the Woodbury terms of <(K~^{-1})_bb, dA_ell>, <., dA_kappa>, tr
  if (threadIdx.x != 0) return;
  const double tr = acc[2] - acc[11];
  const double gt2 = 0.5 * (tr - acc[6]);
  g[3] = gt2;
  g[0] = (0.5 * (nr - acc[5]) - t2 * gt2) / s2;
  g[1] = 0.5 * (acc[0] - acc[9] - acc[3]) + acc[7];
  g[2] = 0.5 * (acc[1] - acc[10] - acc[4]) + acc[8];
}

template <class T> void Engine<T>::grad_adjoint(const double* y_nat, double* g_out) {
  if (!built) throw Error(HODLR_EINVAL, "no build");
  if constexpr (sizeof(T) != 8) {
    throw Error(HODLR_ENOTIMPL, "the adjoint route uses the FP64 factors (HODLR_FP64 or HODLR_MIXED_BF16)");
  } else {
    double* alpha = vec_d + N;
    double* acc = res + 280;       // 12 accumulators (res[280..291]); the result goes to res[300..303]
    double* yt = vec_d;
    HODLR_CUDA(cudaMemsetAsync(acc, 0, 12 * sizeof(double), st));
    permute_rows<double, double>(y_nat, Nr, yt, N, d_perm_plain, N, 1, 0, st);
    solve64(yt, N, alpha, N, 1, 0);
    dot_columns<double, double>(N, 1, alpha, N, yt, N, red, st);
    sum_doubles(red, 1, acc + 5, 1, st);
    dot_columns<double, double>(N, 1, alpha, N, alpha, N, red, st);
    sum_doubles(red, 1, acc + 6, 1, st);
    double* P = (double*)WZ;
    double* Z = (double*)WP;
    // leaves
    adj_leaf_quad_kernel<T><<<nleaves, 256, 0, st>>>(leaf, alpha, dA[0], dA[1], red);
    check_launch("adj_leaf_quad");
    for (int k = 0; k < 2; ++k) sum_doubles_strided_on(red + k, nleaves, 2, acc + 3 + k, st);
    // leaf blocks of K~^{-1}: A_b^{-1} minus the Woodbury terms of every level
    adj_leaf_inv_kernel<T><<<nleaves, 256, 0, st>>>(leaf, d_leafreal, Ainv, dA[0], dA[1], red);
    check_launch("adj_leaf_inv");
    for (int k = 0; k < 3; ++k) sum_doubles_strided_on(red + k, nleaves, 3, acc + k, st);
    for (int l = 1; l <= tau; ++l) {
      const int wl = w[l];
      if (wl == 0) continue;
      double* T1 = P;                                  // M_b U_l[b], N x wl (leaf rows per leaf)
      double* Gb = Z;                                  // U_l[b]^T M_b U_l[b], wl x wl per leaf
      for (int k = 0; k < 3; ++k) {                    // M = dA_ell, dA_kappa, I
        const double* R = U[l];
        if (k < 2) {
          GemmArgs g;
          g.M = leaf; g.N = wl; g.K = leaf;
          g.A = dA[k]; g.lda = leaf; g.sA = (long long)leaf * leaf;
          g.B = U[l]; g.ldb = N; g.sB = leaf;
          g.C = T1; g.ldc = N; g.sC = leaf; g.batch = nleaves;
          g64<T, double>(g);
          R = T1;
        }
        GemmArgs h;
        h.M = wl; h.N = wl; h.K = leaf;
        h.A = U[l]; h.lda = N; h.sA = leaf; h.tA = 1;
        h.B = R; h.ldb = N; h.sB = leaf;
        h.C = Gb; h.ldc = wl; h.sC = (long long)wl * wl; h.batch = nleaves;
        g64<double, double>(h);
        adj_cp_kernel<<<nleaves, 256, 0, st>>>(leaf, wl, msize(l), CP64[l], Gb, red);
        check_launch("adj_cp");
        sum_doubles_strided_on(red, nleaves, 1, acc + 9 + k, st);   // subtracted at the end
      }
    }
    // sibling pairs of every level: the K~^{-1} blocks of the own level and of every coarser one
    const size_t blk = (size_t)nleaves * cap * cap;    // one wp x wl product per child block
    const size_t room = (size_t)N * wide * sizeof(T) / sizeof(double);   // doubles in each wide panel
    if (2 * blk > room || blk + 3 * (size_t)nleaves * cap > room)
      throw Error(HODLR_ENOTIMPL, "adjoint route: the rank cap is too large for the wide panels");
    double* Ab = P;
    double* B0 = P + blk;
    double* B1 = Z;
    for (int l = 1; l <= tau; ++l) {
      const int wl = w[l];
      if (wl == 0) continue;
      const long long m = msize(l);
      const int nb = 1 << l, np = npairs(l);
      auto prod = [&](const double* Ul, int wp, const T* R, double* out) {   // U_l'[c]^T R[c] per child c
        GemmArgs g;
        g.M = wp; g.N = wl; g.K = (int)m;
        g.A = Ul; g.lda = N; g.sA = m; g.tA = 1;
        g.B = R; g.ldb = N; g.sB = m;
        g.C = out; g.ldc = wp; g.sC = (long long)wp * wl; g.batch = nb;
        g64<double, T>(g);
      };
      for (int lp = 1; lp <= l; ++lp) {
        const int wp = w[lp];
        if (wp == 0) continue;
        prod(U[lp], wp, F[l], Ab);
        prod(U[lp], wp, dF[0][l], B0);
        prod(U[lp], wp, dF[1][l], B1);
        adj_pair_kernel<<<np, 256, 0, st>>>(wp, wl, lp == l, m, msize(lp), CP64[lp], Ab, B0, B1, red);
        check_launch("adj_pair");
        for (int k = 0; k < 2; ++k) sum_doubles_strided_on(red + k, np, 2, acc + 7 + k, st);
      }
      // the alpha alpha^T part: a_c = F_l[c]^T alpha_c, b_c = dF_j,l[c]^T alpha_c
      {
        double* av = Z + blk;
        double* bv0 = av + (size_t)nb * wl;
        double* bv1 = bv0 + (size_t)nb * wl;
        auto vec = [&](const T* R, double* out) {
          GemmArgs g;
          g.M = wl; g.N = 1; g.K = (int)m;
          g.A = R; g.lda = N; g.sA = m; g.tA = 1;
          g.B = alpha; g.ldb = N; g.sB = m;
          g.C = out; g.ldc = wl; g.sC = wl; g.batch = nb;
          g64<T, double>(g);
        };
        vec(F[l], av);
        vec(dF[0][l], bv0);
        vec(dF[1][l], bv1);
        adj_alpha_kernel<<<np, 256, 0, st>>>(wl, av, bv0, bv1, red);
        check_launch("adj_alpha");
        for (int k = 0; k < 2; ++k) sum_doubles_strided_on(red + k, np, 2, acc + 7 + k, st);
      }
    }
    double* gd = res + 300;
    adj_finish_kernel<<<1, 32, 0, st>>>(acc, (double)Nr, theta_built[0], theta_built[3], gd);
    check_launch("adj_finish");
    HODLR_CUDA(cudaMemcpyAsync(g_out, gd, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    HODLR_CUDA(cudaStreamSynchronize(st));
  }
}

template struct Engine<double>;
template struct Engine<float>;

}  // namespace hodlr

// ================================================================================ C ABI
using namespace hodlr;

struct hodlr_ctx {
  Base* e = nullptr;
  std::string err;
};

template <class F> static int guarded(hodlr_ctx* h, F f) {
  if (!h || !h->e) return HODLR_EINVAL;
  struct OzScope {   // the context's product path for this call, on this thread
    Base* e;
    explicit OzScope(Base* b) : e(b) { e->oz_enter(true); }
    ~OzScope() { e->oz_enter(false); }
  } scope(h->e);
  try {
    f();
    if (h->e->uses_slices)
      if (int t = oz_status_take(h->e->stream())) throw Error(t, "a tensor-core product gave up waiting for its operands");
    h->err.clear();
    return HODLR_OK;
  } catch (const Error& x) {
    h->err = x.what();
    cudaGetLastError();
    return x.code;
  } catch (const std::bad_alloc& x) {
    h->err = x.what();
    return HODLR_ENOMEM;
  } catch (const std::exception& x) {
    h->err = x.what();
    return HODLR_EINVAL;
  }
}

static Base* make_engine(const hodlr_model* m, const hodlr_opts* o, cudaStream_t st) {
  if (m->precision == HODLR_FP64 || m->precision == HODLR_MIXED_BF16) return new Engine<double>(m, o, st);
  if (m->precision == HODLR_MIXED_FP32) return new Engine<float>(m, o, st);
  throw Error(HODLR_EINVAL, "precision");
}

template <class T> static size_t plan_bytes(Engine<T>* e) {
  Arena ar;
  ar.plan = true;
  e->carve(ar);
  return ar.off + 4096;
}

extern "C" {

size_t hodlr_workspace_size(const hodlr_model* m, const hodlr_opts* o) {
  if (!m || !o) return 0;
  try {
    Base* b = make_engine(m, o, nullptr);
    size_t s = 0;
    if (auto* d = dynamic_cast<Engine<double>*>(b)) s = plan_bytes(d);
    else if (auto* f = dynamic_cast<Engine<float>*>(b)) s = plan_bytes(f);
    delete b;
    return s;
  } catch (...) {
    return 0;
  }
}

int hodlr_plan(const hodlr_model* m, const hodlr_opts* o, int64_t* dims_out, int64_t* perm_out) {
  if (!m || !o || !dims_out) return HODLR_EINVAL;
  try {
    // the engine's constructor builds the tree on the host and touches no device
    std::unique_ptr<Base> b(make_engine(m, o, nullptr));
    dims_out[0] = b->Nr; dims_out[1] = b->tau; dims_out[2] = b->leaf; dims_out[3] = b->c; dims_out[4] = b->cap;
    dims_out[5] = b->nleaves;
    if (perm_out) b->plan_perm(perm_out);
  } catch (const Error& x) {
    return x.code;
  } catch (const std::bad_alloc&) {
    return HODLR_ENOMEM;
  } catch (...) {
    return HODLR_EINVAL;
  }
  return HODLR_OK;
}

int hodlr_create(hodlr_ctx** out, const hodlr_model* m, const hodlr_opts* o, void* cuda_stream, void* workspace,
                 size_t workspace_bytes) {
  if (!out || !m || !o) return HODLR_EINVAL;
  *out = nullptr;
  hodlr_ctx* h = new (std::nothrow) hodlr_ctx;
  if (!h) return HODLR_ENOMEM;
  try {
    h->e = make_engine(m, o, (cudaStream_t)cuda_stream);
    static std::atomic<uint64_t> next_serial{1};
    h->e->serial = next_serial++;
    Arena ar;
    ar.plan = false;
    ar.base = (char*)workspace;
    ar.cap = workspace_bytes;
    if (!workspace || ((uintptr_t)workspace & 255)) throw Error(HODLR_EINVAL, "workspace must be 256-byte aligned");
    if (auto* d = dynamic_cast<Engine<double>*>(h->e)) { d->carve(ar); d->upload_tree(); }
    else if (auto* f = dynamic_cast<Engine<float>*>(h->e)) { f->carve(ar); f->upload_tree(); }
  } catch (const Error& x) {
    int code = x.code;
    delete h->e;
    delete h;
    return code;
  } catch (...) {
    delete h->e;
    delete h;
    return HODLR_EINVAL;
  }
  *out = h;
  return HODLR_OK;
}

int hodlr_build(hodlr_ctx* h, const double* theta, const double* points) {
  if (points) return HODLR_ENOTIMPL;
  if (!theta) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->build(theta); });
}
int hodlr_nll(hodlr_ctx* h, const double* theta, const double* y, double* nll_out) {
  if (!theta || !y || !nll_out) return HODLR_EINVAL;
  return guarded(h, [&] { double v; h->e->eval(theta, y, &v, nullptr, nullptr); *nll_out = v; });
}
int hodlr_grad(hodlr_ctx* h, const double* theta, const double* y, double* grad_out) {
  if (!theta || !y || !grad_out) return HODLR_EINVAL;
  return guarded(h, [&] { double g[4]; h->e->eval(theta, y, nullptr, g, nullptr); std::memcpy(grad_out, g, sizeof(g)); });
}
int hodlr_grad_adjoint(hodlr_ctx* h, const double* theta, const double* y, double* grad_out) {
  if (!theta || !y || !grad_out) return HODLR_EINVAL;
  return guarded(h, [&] {
    double v;
    h->e->eval(theta, y, &v, nullptr, nullptr);   // build and factor at theta (reused when current)
    h->e->grad_adjoint(y, grad_out);
  });
}
int hodlr_fisher(hodlr_ctx* h, const double* theta, double* fisher_out) {
  if (!theta || !fisher_out) return HODLR_EINVAL;
  return guarded(h, [&] { double f[16]; h->e->eval(theta, nullptr, nullptr, nullptr, f); std::memcpy(fisher_out, f, sizeof(f)); });
}
int hodlr_eval(hodlr_ctx* h, const double* theta, const double* y, double* nll_out, double* grad_out,
               double* fisher_out) {
  if (!theta) return HODLR_EINVAL;
  return guarded(h, [&] {
    double v, g[4], f[16];
    h->e->eval(theta, y, nll_out ? &v : nullptr, grad_out ? g : nullptr, fisher_out ? f : nullptr);
    if (nll_out) *nll_out = v;
    if (grad_out) std::memcpy(grad_out, g, sizeof(g));
    if (fisher_out) std::memcpy(fisher_out, f, sizeof(f));
  });
}
}  // extern "C"

namespace {
// One CUDA graph holding the NLL and gradient evaluations of a list of contexts: every
// context's evaluation is captured on a branch stream of its own (forked from and joined to the
// first context's stream), so that the evaluations of small datasets run side by side, and the
// whole list replays as one graph launch.  Cached for the last (contexts, theta, y) list.
struct BatchGraph {
  std::vector<uint64_t> serial;
  std::vector<double> theta;
  std::vector<const double*> y;
  cudaStream_t root = nullptr;              // the library's own stream: graphs are captured and
                                             // launched there, ordered after / before the contexts'
  cudaGraphExec_t exec = nullptr;
  long long nkernels = 0;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;   // ev[0] fork, ev[1 + i] join of branch i
  ~BatchGraph() { reset(); }
  void reset() {
    if (exec) cudaGraphExecDestroy(exec);
    exec = nullptr;
    serial.clear();
  }
  void ensure_resources(int nb) {
    if (!root) HODLR_CUDA(cudaStreamCreateWithFlags(&root, cudaStreamNonBlocking));
    while ((int)br.size() < nb) {
      cudaStream_t s;
      HODLR_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
      br.push_back(s);
    }
    while ((int)ev.size() < nb + 2) {
      cudaEvent_t e;
      HODLR_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      ev.push_back(e);
    }
  }
};
BatchGraph g_batch;
std::mutex g_batch_mu;

void batch_capture(hodlr_ctx* const* hs, int nb, const double* thetas, const double* const* ys) {
  BatchGraph& B = g_batch;
  B.reset();
  std::vector<cudaStream_t> saved(nb);
  for (int i = 0; i < nb; ++i) {
    saved[i] = hs[i]->e->stream();
    hs[i]->e->set_graph_mode(true);
  }
  auto restore = [&] {
    for (int i = 0; i < nb; ++i) {
      hs[i]->e->set_stream(saved[i]);
      hs[i]->e->set_graph_mode(false);   // the next single call rebuilds in the ordinary mode
    }
  };
  const long long k0 = g_kernel_launches;
  cudaGraph_t graph = nullptr;
  // branches: datasets are dealt round-robin to nbr streams (each runs its datasets one after
  // another), so that independent evaluations overlap without flooding the GPU with streams
  int nbr = std::min(nb, 8);
  if (const char* v = getenv("HODLR_BATCH_BRANCHES")) nbr = std::max(1, std::min(nb, atoi(v)));
  HODLR_CUDA(cudaStreamBeginCapture(B.root, cudaStreamCaptureModeRelaxed));
  try {
    HODLR_CUDA(cudaEventRecord(B.ev[0], B.root));
    for (int k = 0; k < nbr; ++k) HODLR_CUDA(cudaStreamWaitEvent(B.br[k], B.ev[0], 0));
    for (int i = 0; i < nb; ++i) {
      hs[i]->e->set_stream(B.br[i % nbr]);
      hs[i]->e->oz_enter(true);
      hs[i]->e->eval_graph(thetas + 4 * (size_t)i, ys[i]);
      hs[i]->e->oz_enter(false);
    }
    for (int k = 0; k < nbr; ++k) {
      HODLR_CUDA(cudaEventRecord(B.ev[1 + k], B.br[k]));
      HODLR_CUDA(cudaStreamWaitEvent(B.root, B.ev[1 + k], 0));
    }
  } catch (...) {
    cudaStreamEndCapture(B.root, &graph);
    if (graph) cudaGraphDestroy(graph);
    restore();
    throw;
  }
  cudaError_t e = cudaStreamEndCapture(B.root, &graph);
  restore();
  if (e != cudaSuccess) throw Error(HODLR_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  e = cudaGraphInstantiate(&B.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    B.exec = nullptr;
    throw Error(HODLR_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  B.nkernels = g_kernel_launches - k0;
  g_kernel_launches = k0;
  for (int i = 0; i < nb; ++i) B.serial.push_back(hs[i]->e->serial);
  B.theta.assign(thetas, thetas + 4 * (size_t)nb);
  B.y.assign(ys, ys + nb);
}
}  // namespace

extern "C" {

int hodlr_batch_nll_grad(hodlr_ctx* const* hs, int nb, const double* thetas, const double* const* ys, double* nll_out,
                         double* grad_out) {
  if (!hs || nb <= 0 || !thetas || !ys || !nll_out || !grad_out) return HODLR_EINVAL;
  for (int i = 0; i < nb; ++i) {
    if (!hs[i] || !hs[i]->e || !ys[i]) return HODLR_EINVAL;
    for (int k = 0; k < 4; ++k)
      if (!(thetas[4 * i + k] > 0.0) || !std::isfinite(thetas[4 * i + k])) return HODLR_EINVAL;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return HODLR_EINVAL;   // one branch per context
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchGraph& B = g_batch;
  std::vector<double> out(6 * (size_t)nb);
  int rc = HODLR_OK;
  try {
    B.ensure_resources(nb);
    bool same = B.exec && (int)B.serial.size() == nb;
    for (int i = 0; same && i < nb; ++i) same = B.serial[i] == hs[i]->e->serial && B.y[i] == ys[i];
    for (int k = 0; same && k < 4 * nb; ++k) same = B.theta[k] == thetas[k];
    if (!same) batch_capture(hs, nb, thetas, ys);
    // the graph runs after the work already queued on the contexts' streams (y, for instance) ...
    cudaEvent_t order = B.ev[nb + 1];
    for (int i = 0; i < nb; ++i) {
      HODLR_CUDA(cudaEventRecord(order, hs[i]->e->stream()));
      HODLR_CUDA(cudaStreamWaitEvent(B.root, order, 0));
    }
    HODLR_CUDA(cudaGraphLaunch(B.exec, B.root));
    // ... and before the work queued on them later
    HODLR_CUDA(cudaEventRecord(order, B.root));
    for (int i = 0; i < nb; ++i) HODLR_CUDA(cudaStreamWaitEvent(hs[i]->e->stream(), order, 0));
    g_kernel_launches += B.nkernels;
    for (int i = 0; i < nb; ++i)
      HODLR_CUDA(cudaMemcpyAsync(out.data() + 6 * (size_t)i, hs[i]->e->graph_out(), 6 * sizeof(double),
                                 cudaMemcpyDeviceToHost, B.root));
    HODLR_CUDA(cudaStreamSynchronize(B.root));
    if (tc_status_take(B.root) || oz_status_take(B.root))
      throw Error(HODLR_ETIMEOUT, "a tensor-core product gave up waiting for its operands");
    for (int i = 0; i < nb && rc == HODLR_OK; ++i)
      if (out[6 * (size_t)i + 5] != 0.0) {
        rc = (int)out[6 * (size_t)i + 5];
        hs[i]->err = "batched evaluation: a Cholesky factorization failed or a result is not finite";
      }
  } catch (const Error& x) {
    hs[0]->err = x.what();
    B.reset();
    return x.code;
  } catch (const std::bad_alloc&) {
    B.reset();
    return HODLR_ENOMEM;
  }
  if (rc != HODLR_OK) return rc;
  for (int i = 0; i < nb; ++i) {
    nll_out[i] = out[6 * (size_t)i];
    for (int j = 0; j < 4; ++j) grad_out[4 * (size_t)i + j] = out[6 * (size_t)i + 1 + j];
  }
  return HODLR_OK;
}
int hodlr_autotune(hodlr_ctx* h, int enable) {
  if (!h || !h->e) return HODLR_EINVAL;
  h->e->tune = enable != 0;
  return HODLR_OK;
}
int hodlr_autotune_clear(void) {
  oz_tuned_clear();
  return HODLR_OK;
}
int hodlr_autotune_table(int64_t* out, int cap, int* n_out) {
  if (!n_out || cap < 0 || (cap > 0 && !out)) return HODLR_EINVAL;
  *n_out = oz_tuned_table(out, cap);
  return HODLR_OK;
}
int hodlr_perm(const hodlr_ctx* h, int64_t* perm_out) {
  if (!h || !h->e || !perm_out) return HODLR_EINVAL;
  try {
    h->e->read_perm(perm_out);
  } catch (const Error& x) {
    return x.code;
  }
  return HODLR_OK;
}
int hodlr_dims(const hodlr_ctx* h, int64_t* out) {
  if (!h || !h->e || !out) return HODLR_EINVAL;
  out[0] = h->e->Nr; out[1] = h->e->tau; out[2] = h->e->leaf; out[3] = h->e->c; out[4] = h->e->cap;
  out[5] = h->e->nleaves;
  return HODLR_OK;
}
int hodlr_ranks(const hodlr_ctx* h, int32_t* ranks_out) {
  if (!h || !h->e || !ranks_out) return HODLR_EINVAL;
  size_t off = 0;
  for (int l = 1; l <= h->e->tau; ++l) {
    const auto& r = h->e->host_rank[l];
    for (size_t p = 0; p < (size_t)(1 << (l - 1)); ++p) ranks_out[off++] = p < r.size() ? r[p] : 0;
  }
  return HODLR_OK;
}
int hodlr_get_pivots(const hodlr_ctx* h, int32_t* piv_out) {
  if (!h || !h->e || !piv_out) return HODLR_EINVAL;
  try { h->e->get_pivots(piv_out); } catch (const Error& x) { return x.code; }
  return HODLR_OK;
}
int hodlr_set_pivots(hodlr_ctx* h, const int32_t* piv_in) {
  return guarded(h, [&] { h->e->set_pivots(piv_in); });
}
int hodlr_apply(hodlr_ctx* h, const double* theta, int which, const double* X, double* Yo, int ncols) {
  if (!theta || !X || !Yo || ncols < 0 || which < 0 || which > 4) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->apply_nat(theta, which, X, Yo, ncols); });
}
int hodlr_probe(hodlr_ctx* h, int level, int ncols, double* out) {
  if (!out) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->probe(level, ncols, out); });
}
int hodlr_densify(hodlr_ctx* h, int which, double* out) {
  if (!out || which < 0 || which > 4) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->densify(which, out); });
}
int hodlr_matvec(hodlr_ctx* h, int which, const double* X, double* Y, int ncols) {
  if (!X || !Y || which < 0 || which > 4 || ncols < 0) return HODLR_EINVAL;
  if (ncols == 0) return HODLR_OK;
  return guarded(h, [&] { h->e->matvec_nat(which, X, Y, ncols); });
}
int hodlr_solve(hodlr_ctx* h, const double* b, double* x) {
  if (!b || !x) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->solve_nat(b, x); });
}
int hodlr_logdet(hodlr_ctx* h, double* logdet_out) {
  if (!logdet_out) return HODLR_EINVAL;
  return guarded(h, [&] {
    if (!h->e->built) throw Error(HODLR_EINVAL, "no build");
    *logdet_out = h->e->logdet;
  });
}
int hodlr_traces(hodlr_ctx* h, double* t_out, double* f_out) {
  if (!t_out || !f_out) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->traces(t_out, f_out); });
}
int hodlr_debug_level(hodlr_ctx* h, int what, int level, double* out, int64_t count, int32_t* w_out) {
  if (!out || !w_out || what < 0 || what > 3) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->debug_level(what, level, out, count, w_out); });
}
int hodlr_logdet_levels(hodlr_ctx* h, double* out) {
  if (!out) return HODLR_EINVAL;
  return guarded(h, [&] { h->e->logdet_levels(out); });
}
int hodlr_napply(const hodlr_ctx* h, int64_t* out) {
  if (!h || !h->e || !out) return HODLR_EINVAL;
  *out = h->e->napply;
  return HODLR_OK;
}
int hodlr_profile(hodlr_ctx* h, int enable) {
  if (!h || !h->e) return HODLR_EINVAL;
  try {
    if (!g_prof.ev) {
      g_prof.cap = 65536;
      g_prof.ev = new cudaEvent_t[2 * g_prof.cap];
      g_prof.shape = new int[7 * g_prof.cap];
      for (int i = 0; i < 2 * g_prof.cap; ++i) HODLR_CUDA(cudaEventCreate(&g_prof.ev[i]));
    }
    g_prof.n = 0;
    g_prof.flops = g_prof.bytes = 0.0;
    for (double& b : g_prof.fbytes) b = 0.0;
    g_prof.on = enable != 0;
    g_trace.on = false;
    if (enable && getenv("HODLR_TRACE")) {
      if (!g_trace.ev) {
        g_trace.cap = 200000;
        g_trace.ev = new cudaEvent_t[g_trace.cap + 1];
        g_trace.name = new const char*[g_trace.cap];
        for (int i = 0; i <= g_trace.cap; ++i) HODLR_CUDA(cudaEventCreate(&g_trace.ev[i]));
      }
      g_trace.n = 0;
      g_trace.stream = h->e->stream();
      HODLR_CUDA(cudaEventRecord(g_trace.ev[0], g_trace.stream));
      g_trace.on = true;
    }
  } catch (const Error& x) {
    h->err = x.what();
    return x.code;
  } catch (const std::exception& x) {   // host allocation of the event tables
    h->err = x.what();
    return HODLR_ENOMEM;
  }
  return HODLR_OK;
}
int hodlr_profile_read(hodlr_ctx* h, double* out) {
  if (!h || !h->e || !out) return HODLR_EINVAL;
  try {
    double ms = 0.0;
    double per[8][3] = {{0}};   // per kernel family: ms, flops, launches
    for (int i = 0; i < g_prof.n; ++i) {
      HODLR_CUDA(cudaEventSynchronize(g_prof.ev[2 * i + 1]));
      float t = 0.f;
      HODLR_CUDA(cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]));
      ms += t;
      const int* sh = g_prof.shape + 7 * i;
      const int v = prof_family(sh[6]);
      per[v][0] += t;
      per[v][1] += 2.0 * (double)sh[0] * sh[1] * sh[2] * sh[3];
      per[v][2] += 1.0;
    }
    out[0] = ms;
    out[1] = g_prof.n;
    for (int v = 0; v < 8; ++v) {
      for (int k = 0; k < 3; ++k) out[4 + 4 * v + k] = per[v][k];
      out[7 + 4 * v] = g_prof.fbytes[v];
    }
    // optional per-launch dump (shape and time) for kernel studies
    if (const char* path = getenv("HODLR_PROFILE_DUMP")) {
      if (FILE* f = fopen(path, "w")) {
        fprintf(f, "M,N,K,batch,tA,tB,variant,ms\n");
        for (int i = 0; i < g_prof.n; ++i) {
          float t = 0.f;
          cudaEventElapsedTime(&t, g_prof.ev[2 * i], g_prof.ev[2 * i + 1]);
          const int* sh = g_prof.shape + 7 * i;
          fprintf(f, "%d,%d,%d,%d,%d,%d,%d,%.6f\n", sh[0], sh[1], sh[2], sh[3], sh[4], sh[5], sh[6], t);
        }
        fclose(f);
      }
    }
    out[2] = g_prof.flops;
    out[3] = g_prof.bytes;
    // optional launch timeline, summed per launcher name
    if (const char* path = getenv("HODLR_TRACE")) {
      if (g_trace.n > 0) {
        HODLR_CUDA(cudaEventSynchronize(g_trace.ev[g_trace.n]));
        std::map<std::string, std::pair<long long, double>> agg;
        for (int i = 0; i < g_trace.n; ++i) {
          float t = 0.f;
          HODLR_CUDA(cudaEventElapsedTime(&t, g_trace.ev[i], g_trace.ev[i + 1]));
          auto& a = agg[g_trace.name[i]];
          a.first += 1;
          a.second += t;
        }
        if (FILE* f = fopen(path, "w")) {
          fprintf(f, "name,launches,ms\n");
          for (auto& kv : agg) fprintf(f, "%s,%lld,%.6f\n", kv.first.c_str(), kv.second.first, kv.second.second);
          fclose(f);
        }
      }
      g_trace.on = false;
    }
  } catch (const Error& x) {
    h->err = x.what();
    return x.code;
  }
  return HODLR_OK;
}
int hodlr_kernel_count(const hodlr_ctx* h, int64_t* out) {
  if (!h || !out) return HODLR_EINVAL;
  *out = g_kernel_launches;
  return HODLR_OK;
}
int hodlr_reset_kernel_count(hodlr_ctx* h) {
  if (!h) return HODLR_EINVAL;
  g_kernel_launches = 0;
  return HODLR_OK;
}
int hodlr_debug_wait_limit(int polls) { return tc_set_first_wait_limit(polls); }
const char* hodlr_last_error(const hodlr_ctx* h) { return h ? h->err.c_str() : "null context"; }
void hodlr_destroy(hodlr_ctx* h) {
  if (!h) return;
  delete h->e;
  delete h;
}

}  // extern "C"
