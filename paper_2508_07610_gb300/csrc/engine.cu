// Host engine behind the C ABI: owns the device state of a batch of MPDO chains and sequences the
// sm_103a kernels for each call.  Shapes are decided on the host from the gate sequence alone, so
// no call reads device data to size its work and whole circuits can be captured in a CUDA graph.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <new>
#include <type_traits>
#include <vector>

#include "kernels.h"
#include "mpdo.h"

using namespace mpdo;

struct mpdo_chanset {
  int nq = 0, count = 0, rpad = 0;
  int device = 0;
  cplx<double>* kraus = nullptr;  // [count][rpad][d][d]
  std::vector<int> ranks;
  ~mpdo_chanset() {
    if (kraus) cudaFree(kraus);
  }
};

struct mpdo_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;
  ~mpdo_graph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
  }
};

#define CK(x)                                                        \
  do {                                                               \
    cudaError_t e_ = (x);                                            \
    if (e_ != cudaSuccess) {                                         \
      last_err = e_;                                                 \
      return e_ == cudaErrorInvalidValue ? MPDO_EINVAL : MPDO_ECUDA; \
    }                                                                \
  } while (0)

namespace {

inline int imin(int a, int b) { return a < b ? a : b; }
inline int64_t lmax(int64_t a, int64_t b) { return a > b ? a : b; }

View v2(int64_t bstride, int32_t rdiv, int64_t rhi, int64_t rlo, int32_t cdiv, int64_t chi, int64_t clo, int conj = 0) {
  View v{};
  v.blo = bstride;
  v.rdiv = rdiv;
  v.rhi = rhi;
  v.rlo = rlo;
  v.cdiv = cdiv;
  v.chi = chi;
  v.clo = clo;
  v.conj = conj;
  return v;
}

struct EngBase {
  int B = 1, n = 0, chi_max = 1, kappa_max = 1, prec = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  bool capturing = false;
  long long launches = 0;
  cudaError_t last_err = cudaSuccess;
  std::vector<int> bond;   // n + 1 entries, bond[0] = bond[n] = 1
  std::vector<int> kraus;  // n entries
  int centre = 0;
  // A site next to the centre whose Kraus leg was truncated through the centre's environment (so it
  // is not isometric); -1 when every site other than the centre is isometric.
  int dirty = -1;
  bool neighbour_trunc = false;  // let 1q gates on a neighbour of the centre skip the centre move
  int64_t purity_limit = 0;      // bytes for the purity chunk buffers, 0 = a share of free memory
  bool tensor_cores = false;     // complex64 products that qualify run on the tcgen05 GEMM
  int trunc_order = MPDO_TRUNC_SPLIT_FIRST;  // order of the bond split and the Kraus-leg truncation
  // capture snapshot
  std::vector<int> snap_bond, snap_kraus, snap_slot;
  int snap_centre = 0;
  // optional per-launch CUDA-event timing by kernel class (not while capturing)
  enum { P_GEMM = 0, P_QR = 1, P_EIG = 2, P_OTHER = 3, P_GEMM_GRAM = 4, P_GEMM_X = 5, P_EIG_BOND = 6,
         P_EIG_KRAUS = 7, P_ONEQ = 8, P_N = 9 };
  int prof_sub = -1;  // sub-class (one call site) of the next profiled launch, -1 = none
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec {
    int cls, sub;
    int e0, e1;
    double flops, bytes;
  };
  std::vector<Rec> recs;
  int ev_next = 0;
  int cur_cls = -1, cur_sub = -1, cur_e0 = -1;
  double cur_flops = 0, cur_bytes = 0;
  double prof_bytes = 0;  // algorithmic bytes of the next profiled launch (HBM-bound call sites)
  void prof_start(int cls, double flops) {
    if (!prof_on || capturing) return;
    if (ev_next + 2 > (int)ev_pool.size()) return;
    cur_cls = cls;
    cur_sub = prof_sub;
    cur_flops = flops;
    cur_bytes = prof_bytes;
    cur_e0 = ev_next++;
    cudaEventRecord(ev_pool[cur_e0], stream);
  }
  void prof_stop() {
    if (cur_cls < 0) return;
    int e1 = ev_next++;
    cudaEventRecord(ev_pool[e1], stream);
    recs.push_back({cur_cls, cur_sub, cur_e0, e1, cur_flops, cur_bytes});
    cur_cls = -1;
  }

  // algorithmic real flops (LAPACK operation counts, complex arithmetic = 4 real per multiply and add):
  // Householder QR of an m x n matrix with the thin Q formed, p = min(m, n)
  static double qr_flops(int m, int n) {
    const double M = m > n ? m : n, P = m < n ? m : n;
    return 2.0 * 8.0 * (M * P * P - P * P * P / 3.0);
  }
  // Hermitian eigenproblem of order n, k vectors: tridiagonalisation + back-transformation
  static double eig_flops(int n, int k) {
    const double N = n;
    return (16.0 / 3.0) * N * N * N + 8.0 * N * N * k;
  }

  virtual ~EngBase() {
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  }
  virtual mpdo_status alloc() = 0;
  virtual mpdo_status reset() = 0;
  virtual mpdo_status apply(int nq, int q, const double* Uhost, const double* Udev, const mpdo_chanset* ch,
                            const int* idx_dev) = 0;
  virtual mpdo_status truncate(int q, int kappa, double* disc) = 0;
  virtual mpdo_status truncate_bonds(int chi, double* disc) = 0;
  virtual mpdo_status expect(int kind, const int* args, int nargs, double* out) = 0;
  virtual mpdo_status restore_layout() = 0;
  virtual std::vector<int> slots() const = 0;
  virtual mpdo_status clean() = 0;
  virtual mpdo_status save(FILE* f) = 0;
  virtual mpdo_status get_site(int chain, int q, double* out) = 0;
  virtual mpdo_status set_site(int q, int dl, int dn, int dr, const double* data) = 0;
  virtual mpdo_status load(FILE* f) = 0;
  virtual mpdo_status alloc_tc() = 0;
  // dense density matrix of one chain (small n), FP64, see Eng::dense_rho
  virtual int64_t dense_work() const = 0;
  virtual mpdo_status distribution(double* out) = 0;
  virtual mpdo_status dense_rho(int chain, cudaStream_t s, cplx<double>* X, cplx<double>* Y, cplx<double>* S) = 0;

  int* dStatus = nullptr;  // device status word: kStatusNoConv | kStatusTimeout bits set by kernels

  mpdo_status sync() {
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
      last_err = e;
      return MPDO_ECUDA;
    }
    return read_status();
  }
  // Synchronises, reads the status word and clears it: a bounded wait that ran out is reported as
  // MPDO_ETIMEOUT, an eigensolver that produced non-finite or collapsed eigenpairs as MPDO_ENOCONV.
  mpdo_status read_status() {
    if (!dStatus) return MPDO_OK;
    int h = 0;
    cudaError_t e = cudaMemcpyAsync(&h, dStatus, sizeof(int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && h) e = cudaMemsetAsync(dStatus, 0, sizeof(int), stream);
    if (e != cudaSuccess) {
      last_err = e;
      return MPDO_ECUDA;
    }
    if (h & kStatusTimeout) return MPDO_ETIMEOUT;
    if (h & kStatusNoConv) return MPDO_ENOCONV;
    return MPDO_OK;
  }
};

template <typename R, typename ER>
struct Eng : EngBase {
  using C = cplx<R>;
  using CE = cplx<ER>;
  static constexpr int RMAX = 16;

  // storage
  C* pool = nullptr;
  int nslots = 0;
  int64_t slot_elems = 0;
  std::vector<int> site_slot, free_slots;
  // per-instance workspaces (each strided by its own size)
  C *wQR = nullptr, *wQ = nullptr, *wE = nullptr, *wT = nullptr, *wZ = nullptr, *wF = nullptr, *wU = nullptr,
    *wH = nullptr, *wY = nullptr, *wX = nullptr, *wK = nullptr, *wRt = nullptr;
  int64_t sQR = 0, sE = 0, sT = 0, sZ = 0, sF = 0, sU = 0, sH = 0, sY = 0, sX = 0;
  CE *wF64 = nullptr, *wU64 = nullptr;
  ER *wEval = nullptr, *wScr = nullptr;
  C* wSK = nullptr;
  int64_t sSK = 0;
  C* wHk = nullptr;  // Kraus-first update: the Gram H of Theta0 over (x, r), then the folded gate W
  int64_t sHk = 0;
  // three-site update: allocated at the first three-qubit gate of the handle
  C *w3a = nullptr, *w3b = nullptr, *w3c = nullptr, *w3K = nullptr, *w3F = nullptr, *w3U = nullptr;
  CE *w3F64 = nullptr, *w3U64 = nullptr;
  ER *w3Eval = nullptr, *w3Scr = nullptr;
  int64_t s3a = 0, s3b = 0, s3c = 0, s3F = 0, s3Eval = 0, s3Scr = 0;
  // complex64: split operand planes of the tensor-core GEMM (floats, all chains); a product whose
  // planes do not fit runs on the CUDA cores
  float *tcA = nullptr, *tcB = nullptr;
  int64_t tcCapA = 0, tcCapB = 0;
  int64_t sEval = 0, sScr = 0;
  double* dDisc = nullptr;  // [B][3]: chi, kappa, gap
  // readout buffers
  C *envL = nullptr, *envR = nullptr, *tmpA = nullptr, *tmpB = nullptr;
  int64_t sEnv = 0, sTmp = 0;
  cplx<double>* dDot = nullptr;
  // purity buffers (lazy)
  C *pX = nullptr, *pP = nullptr, *pE = nullptr, *pE2 = nullptr;
  int64_t pCap = 0, pECap = 0, pLimit = 0;

  ~Eng() override {
    void* ptrs[] = {pool, wQR, wQ, wE, wT, wZ, wF, wU, wH, wY, wX, wK, wRt, wF64, wU64, wEval, wScr, dDisc, wSK,
                    envL, envR, tmpA, tmpB, dDot, pX, pP, pE, pE2, iota, dStatus, wHk, tcA, tcB,
                    w3a, w3b, w3c, w3K, w3F, w3U, w3F64, w3U64, w3Eval, w3Scr, dExp2};
    for (void* p : ptrs)
      if (p) cudaFree(p);
  }

  template <typename T>
  cudaError_t dmalloc(T** p, int64_t count) {
    return cudaMalloc((void**)p, sizeof(T) * (size_t)lmax(count, 1));
  }

  C* site_ptr(int q) const { return pool + (int64_t)site_slot[q] * B * slot_elems; }
  C* slot_ptr(int s) const { return pool + (int64_t)s * B * slot_elems; }
  int take_slot() {
    int s = free_slots.back();
    free_slots.pop_back();
    return s;
  }
  void give_slot(int s) { free_slots.push_back(s); }

  mpdo_status alloc() override {
    const int64_t X = chi_max, K = kappa_max;
    slot_elems = 2 * K * X * X;
    nslots = n + 3;
    CK(dmalloc(&pool, (int64_t)nslots * B * slot_elems));
    sQR = 2 * K * X * X;
    CK(dmalloc(&wQR, sQR * B));
    CK(dmalloc(&wQ, sQR * B));
    sE = 4 * X * X;
    CK(dmalloc(&wE, sE * B));
    sT = 16 * X * X;
    CK(dmalloc(&wT, sT * B));
    sZ = 16 * X * X;
    CK(dmalloc(&wZ, sZ * B));
    sF = lmax(16 * X * X, 256 * K * K);
    CK(dmalloc(&wF, sF * B));
    sU = lmax(4 * X * X, 16 * K * K);
    CK(dmalloc(&wU, sU * B));
    sH = 4 * X * X;
    CK(dmalloc(&wH, sH * B));
    sY = lmax(4 * X * X * RMAX, 8 * K * X * X);
    CK(dmalloc(&wY, sY * B));
    sX = 2 * RMAX * K * X * X;
    CK(dmalloc(&wX, sX * B));
    CK(dmalloc(&wK, (int64_t)RMAX * 16 * B));
    CK(dmalloc(&wRt, (int64_t)64 * B));
    if (!std::is_same<R, ER>::value) {
      CK(dmalloc(&wF64, sF * B));
      CK(dmalloc(&wU64, sU * B));
    }
    sEval = lmax(4 * X, 16 * K) + 1;
    CK(dmalloc(&wEval, sEval * B));
    sScr = lmax(eig_scratch_elems((int)(4 * X), (int)X), eig_scratch_elems((int)(16 * K), (int)K));
    sScr = lmax(sScr, eig_scratch_elems(16, 16));
    CK(dmalloc(&wScr, sScr * B));
    CK(dmalloc(&dDisc, (int64_t)3 * B));
    sSK = 4 * lmax(256 * K * K, 1024) * B;  // split-K partials of the long Gram products
    CK(dmalloc(&wSK, sSK));
    sEnv = X * X;
    CK(dmalloc(&envL, sEnv * B * (n + 1)));
    CK(dmalloc(&envR, sEnv * B * (n + 1)));
    sTmp = 2 * K * X * X;
    CK(dmalloc(&tmpA, sTmp * B));
    CK(dmalloc(&tmpB, sTmp * B));
    CK(dmalloc(&dDot, (int64_t)B));
    if (!std::is_same<R, double>::value) {
      mpdo_status ts = alloc_tc();
      if (ts) return ts;
      tensor_cores = true;
    }
    CK(dmalloc(&dStatus, 1));
    CK(dmalloc(&dExp2, (int64_t)B));
    sHk = 16 * K * K;
    CK(dmalloc(&wHk, sHk * B));
    CK(cudaMemset(dStatus, 0, sizeof(int)));
    {
      std::vector<int> h(B);
      for (int b = 0; b < B; ++b) h[b] = b;
      CK(dmalloc(&iota, (int64_t)B));
      CK(cudaMemcpy(iota, h.data(), sizeof(int) * B, cudaMemcpyHostToDevice));
    }
    mpdo_status st = reset();
    if (st) return st;
    return sync();
  }

  // Elements of each of the two work buffers dense_rho needs: the largest intermediate of its
  // contraction, 4^q dl (2 dn dr) at site q.
  int64_t dense_work() const override {
    int64_t w = 1;
    for (int q = 0; q < n; ++q) {
      const int64_t M2 = (int64_t)1 << (2 * q);
      w = lmax(w, M2 * bond[q] * 2 * kraus[q] * bond[q + 1]);
      w = lmax(w, M2 * 4 * (int64_t)bond[q + 1] * bond[q + 1]);
    }
    return w;
  }
  // rho of one chain, row-major 2^n x 2^n FP64 in X (basis index with qubit 0 most significant), by
  // the contraction of Sec. II.C site by site: R[(A),(B), l, l'] -> R'[(A a),(B b), r, r'] =
  // sum_{l, l', n} R[A, B, l, l'] T[l, a, n, r] conj(T[l', b, n, r']) as two products with permutes.
  // X, Y: dense_work() elements each; S: one site in FP64 (slot_elems).
  mpdo_status dense_rho(int chain, cudaStream_t s, cplx<double>* X, cplx<double>* Y, cplx<double>* S) override {
    CK(fill<double>(s, 1, X, mk<double>(1, 0)));
    for (int q = 0; q < n; ++q) {
      const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
      const int64_t Mq = (int64_t)1 << q, M2 = Mq * Mq, N1 = 2 * dn * dr;
      CK((convert<R, double>(s, (int64_t)dl * N1, site_ptr(q) + (int64_t)chain * slot_elems, S)));
      GemmArgs<double> g;
      g.alpha = mk<double>(1, 0);
      g.beta = mk<double>(0, 0);
      // Y[(AB, l'), (a, n, r)] = sum_l R[AB, l, l'] S[l, (a, n, r)]
      g.M = (int)(M2 * dl);
      g.N = (int)N1;
      g.K = dl;
      g.A = X;
      g.va = v2(0, dl, (int64_t)dl * dl, 1, 0, 0, dl);
      g.B = S;
      g.vb = row_major(N1, 0);
      g.C = Y;
      g.vc = row_major(N1, 0);
      CK(gemm<double>(s, 1, g));
      // X[AB][a][r][l'][n] from Y[AB][l'][a][n][r]
      {
        int dims[5] = {(int)M2, dl, 2, dn, dr};
        int perm[5] = {0, 2, 4, 1, 3};
        CK(permute<double>(s, 1, 5, dims, perm, Y, 0, X, 0));
      }
      // Y[(AB, a, r), (b, r')] = sum_{(l', n)} X[(AB, a, r), (l', n)] conj(S[l', b, n, r'])
      g.M = (int)(M2 * 2 * dr);
      g.N = 2 * dr;
      g.K = dl * dn;
      g.A = X;
      g.va = row_major((int64_t)dl * dn, 0);
      g.B = S;
      g.vb = v2(0, dn, N1, dr, dr, (int64_t)dn * dr, 1, 1);
      g.C = Y;
      g.vc = row_major(2 * dr, 0);
      CK(gemm<double>(s, 1, g));
      // X[A][a][B][b][r][r'] from Y[A][B][a][r][b][r']
      {
        int dims[6] = {(int)Mq, (int)Mq, 2, dr, 2, dr};
        int perm[6] = {0, 2, 1, 4, 3, 5};
        CK(permute<double>(s, 1, 6, dims, perm, Y, 0, X, 0));
      }
      launches += 6;
    }
    return MPDO_OK;
  }

  // Plane workspaces of the tensor-core GEMM, sized for the largest operands of the update's products
  // at the caps (per chain; the bond split's F' runs with two batch items per chain).
  mpdo_status alloc_tc() override {
    if (std::is_same<R, double>::value || tcA) return MPDO_OK;
    const int X = chi_max, K = kappa_max;
    const int shapes[][2] = {{32 * X, 2 * X}, {16 * K, 2 * X * X}, {4 * X, 2 * X}, {2 * K * X, X}, {K * X, 2 * X},
                             {8 * K * X, X},  {2 * X, K * X},      {8 * X, 2 * X}, {2 * X, 2 * X}, {4 * X, X},
                             {2 * X * X, 4 * K}, {2 * K * X, 4 * X}, {X, 2 * K * X}, {4 * K, 2 * X * X}};
    int64_t a = 0, b = 0;
    for (auto& sh : shapes) {
      a = lmax(a, tc_plane_floats_a(sh[0], sh[1]));
      b = lmax(b, tc_plane_floats_b(sh[0], sh[1]));
    }
    tcCapA = 2 * a * B;
    tcCapB = 2 * b * B;
    cudaError_t e1 = cudaMalloc((void**)&tcA, sizeof(float) * (size_t)tcCapA);
    cudaError_t e2 = e1 == cudaSuccess ? cudaMalloc((void**)&tcB, sizeof(float) * (size_t)tcCapB) : e1;
    if (e1 != cudaSuccess || e2 != cudaSuccess) {
      if (tcA) cudaFree(tcA);
      tcA = nullptr;
      tcCapA = tcCapB = 0;
      last_err = e1 != cudaSuccess ? e1 : e2;
      return MPDO_ENOMEM;
    }
    return MPDO_OK;
  }

  mpdo_status reset() override {
    bond.assign(n + 1, 1);
    kraus.assign(n, 1);
    centre = 0;
    site_slot.resize(n);
    free_slots.clear();
    for (int q = 0; q < n; ++q) site_slot[q] = q;
    for (int s = nslots - 1; s >= n; --s) free_slots.push_back(s);
    // |0> product state: slot q of every chain holds [1, 0]
    CK(init_zero_sites<R>(stream, n * B, pool, slot_elems));
    CK(cudaMemsetAsync(dExp2, 0, sizeof(int) * B, stream));
    CK(init_discarded(stream, B, dDisc));
    launches += 2;
    return MPDO_OK;
  }

  std::vector<int> slots() const override { return site_slot; }
  // make every site other than the centre isometric again (absorbs a non-isometric neighbour)
  mpdo_status clean() override {
    if (dirty < 0) return MPDO_OK;
    return move_centre(dirty);
  }

  // ---------------------------------------------------------------- kernels wrappers
  mpdo_status gemm_(int M, int N, int K, const C* A, View va, const C* Bm, View vb, C* Cm, View vc, int batch = -1,
                    int herm = 0, bool accumulate = false) {
    GemmArgs<R> g;
    g.herm = herm;
    g.allow_tc = tensor_cores ? 1 : 0;
    g.ws = wSK;
    g.ws_elems = sSK;
    g.status = dStatus;
    g.tc_a = tcA;
    g.tc_b = tcB;
    g.tc_a_cap = tcCapA;
    g.tc_b_cap = tcCapB;
    g.M = M;
    g.N = N;
    g.K = K;
    g.alpha = mk<R>(1, 0);
    g.beta = mk<R>(accumulate ? 1 : 0, 0);
    g.A = A;
    g.va = va;
    g.B = Bm;
    g.vb = vb;
    g.C = Cm;
    g.vc = vc;
    const int nb = batch < 0 ? B : batch;
    double frac = 1.0;  // a Hermitian result computes only the tiles on and below the diagonal
    if (herm) {
      const int tile = (M <= 32 && N <= 32) ? 32 : 64;
      double T = (M + tile - 1) / tile;
      frac = (T * (T + 1) / 2) / (T * T);
    }
    prof_start(P_GEMM, 8.0 * M * N * K * nb * frac);
    CK(gemm<R>(stream, nb, g));
    prof_stop();
    ++launches;
    return MPDO_OK;
  }

  // top-k eigenpairs of the column-major Hermitian matrices in wF (n x n), vectors to wU (col-major n x k)
  // Buffers of one eigensolver call: Gram matrices in (F, stride sF), eigenvectors out in (U, sU),
  // their FP64 copies in the complex64 modes, eigenvalues and scratch.
  struct EigBufs {
    C *F, *U;
    int64_t sF, sU;
    CE *F64, *U64;
    ER *eval, *scr;
    int64_t sEval, sScr;
  };
  EigBufs main_bufs() { return {wF, wU, sF, sU, wF64, wU64, wEval, wScr, sEval, sScr}; }

  mpdo_status eig_(int nmat, int k, int which /*0 chi, 1 kappa, -1 none*/, const EigBufs* eb = nullptr) {
    prof_sub = which == 0 ? P_EIG_BOND : which == 1 ? P_EIG_KRAUS : -1;
    const EigBufs b = eb ? *eb : main_bufs();
    mpdo_status st = eig_impl(nmat, k, which, b);
    prof_sub = -1;
    return st;
  }
  mpdo_status eig_impl(int nmat, int k, int which, const EigBufs& b) {
    EigArgs<ER> a;
    a.n = nmat;
    a.k = k;
    a.astride = b.sF;
    a.w = b.eval;
    a.wstride = b.sEval;
    a.vv = col_major(nmat, b.sU);
    a.scratch = b.scr;
    a.sstride = b.sScr;
    a.disc = which >= 0 ? dDisc + which : nullptr;
    a.gap = which >= 0 ? dDisc + 2 : nullptr;
    a.disc_stride = 3;
    a.status = dStatus;
    if (std::is_same<R, ER>::value) {
      a.A = reinterpret_cast<CE*>(b.F);
      a.V = reinterpret_cast<CE*>(b.U);
      prof_start(P_EIG, eig_flops(nmat, k) * B);
      CK(heevk<ER>(stream, B, a));
      prof_stop();
      ++launches;
    } else {
      // FP64 eigensolver on complex64 Gram matrices
      const int sub = prof_sub;
      prof_sub = -1;
      prof_start(P_OTHER, 0);
      CK((convert<R, ER>(stream, b.sF * B, b.F, b.F64)));
      prof_stop();
      prof_sub = sub;
      a.A = b.F64;
      a.V = b.U64;
      prof_start(P_EIG, eig_flops(nmat, k) * B);
      CK(heevk<ER>(stream, B, a));
      prof_stop();
      prof_sub = -1;
      prof_start(P_OTHER, 0);
      CK((convert<ER, R>(stream, b.sU * B, b.U64, b.U)));
      prof_stop();
      prof_sub = sub;
      launches += 3;
    }
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- canonical form
  // centre c -> c + 1: QR of site c as ((l, p, n), r)
  mpdo_status shift_right(int c) {
    const int dl = bond[c], dn = kraus[c], dr = bond[c + 1];
    const int m = dl * 2 * dn, x = imin(m, dr);
    const int dn2 = kraus[c + 1], dr2 = bond[c + 2];
    const int sa = take_slot(), sb = take_slot();
    QrArgs<R> a;
    a.m = m;
    a.n = dr;
    a.in = site_ptr(c);
    a.vin = row_major(dr, slot_elems);
    a.W = wQR;
    a.wstride = sQR;
    a.Qw = wQ;
    a.qstride = sQR;
    a.qout = slot_ptr(sa);
    a.vq = row_major(x, slot_elems);
    prof_start(P_QR, qr_flops(a.m, a.n) * B);
    CK(qr<R>(stream, B, a));
    prof_stop();
    ++launches;
    // site c+1 <- R . A_{c+1}
    const int N = 2 * dn2 * dr2;
    mpdo_status st = gemm_(x, N, dr, wQR, col_major(m, sQR), site_ptr(c + 1), row_major(N, slot_elems),
                           slot_ptr(sb), row_major(N, slot_elems));
    if (st) return st;
    give_slot(site_slot[c]);
    give_slot(site_slot[c + 1]);
    site_slot[c] = sa;
    site_slot[c + 1] = sb;
    bond[c + 1] = x;
    return MPDO_OK;
  }
  // centre c -> c - 1: LQ of site c as (l, (p, n, r)) via QR of its conjugate transpose
  mpdo_status shift_left(int c) {
    const int dl = bond[c], dn = kraus[c], dr = bond[c + 1];
    const int L = 2 * dn * dr, x = imin(L, dl);
    const int dlp = bond[c - 1], dnp = kraus[c - 1];
    const int sa = take_slot(), sb = take_slot();
    QrArgs<R> a;
    a.m = L;
    a.n = dl;
    a.in = site_ptr(c);
    a.vin = v2(slot_elems, 0, 0, 1, 0, 0, L, 1);  // (i, j) -> conj(A[j * L + i])
    a.W = wQR;
    a.wstride = sQR;
    a.Qw = wQ;
    a.qstride = sQR;
    a.qout = slot_ptr(sa);
    a.vq = v2(slot_elems, 0, 0, 1, 0, 0, L, 1);  // Q^H written as the new x x L site
    prof_start(P_QR, qr_flops(a.m, a.n) * B);
    CK(qr<R>(stream, B, a));
    prof_stop();
    ++launches;
    // site c-1 <- A_{c-1} . R^H
    const int M = dlp * 2 * dnp;
    mpdo_status st = gemm_(M, x, dl, site_ptr(c - 1), row_major(dl, slot_elems), wQR, v2(sQR, 0, 0, L, 0, 0, 1, 1),
                           slot_ptr(sb), row_major(x, slot_elems));
    if (st) return st;
    give_slot(site_slot[c]);
    give_slot(site_slot[c - 1]);
    site_slot[c] = sa;
    site_slot[c - 1] = sb;
    bond[c] = x;
    return MPDO_OK;
  }
  mpdo_status move_centre(int q) {
    // the first hop goes onto a non-isometric neighbour, which makes it the centre again
    if (dirty >= 0 && dirty != centre) {
      mpdo_status s = (dirty == centre + 1) ? shift_right(centre) : shift_left(centre);
      if (s) return s;
      centre = dirty;
    }
    dirty = -1;
    while (centre < q) {
      mpdo_status s = shift_right(centre);
      if (s) return s;
      ++centre;
    }
    while (centre > q) {
      mpdo_status s = shift_left(centre);
      if (s) return s;
      --centre;
    }
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- gate fusion
  mpdo_status fuse_(int nq, const double* Uhost, const double* Udev, const mpdo_chanset* ch, const int* idx_dev) {
    FuseArgs<R> f;
    std::memset(&f, 0, sizeof(f));
    f.nq = nq;
    f.rk = ch->rpad;
    const int d = 1 << nq;
    if (Uhost)
      for (int i = 0; i < d * d; ++i) f.U[i] = mk<double>(Uhost[2 * i], Uhost[2 * i + 1]);
    f.Udev = reinterpret_cast<const cplx<double>*>(Udev);
    f.kraus = ch->kraus;
    f.chan_stride = (int64_t)ch->rpad * d * d;
    f.chan_idx = idx_dev;
    f.Khat = nq == 3 ? w3K : wK;
    f.Rt = nq == 2 ? wRt : nullptr;
    // idx_dev == nullptr: one channel for all, or channel b for chain b (handled by chan_idx below)
    prof_start(P_OTHER, 0);
    CK(fuse_gate<R>(stream, B, f));
    prof_stop();
    ++launches;
    return MPDO_OK;
  }

  // Kraus-leg truncation of a tensor held Kraus-major in wX: X[nk][s][r] (NK x S*dr) -> new site
  // [l][p][nu][r] with S = dl*2 rows (l, p).  Eq. (svdNoise) through the Gram matrix X^* X^T.
  // With Yg (same layout as X, stride sY) the Gram is conj(X) Yg^T: Yg carries the environment of a
  // site next to the centre.
  // The three-site update passes its own X buffer (Xs, stride xs) and eigensolver buffers (eb).
  mpdo_status kappa_truncate_X(int NK, int S, int dr, int kap, int out_slot, const C* Yg = nullptr,
                               const C* Xs = nullptr, int64_t xs = 0, const EigBufs* eb = nullptr) {
    const int64_t L = (int64_t)S * dr;
    const C* Xb = Xs ? Xs : wX;
    const int64_t sx = Xs ? xs : sX;
    const EigBufs b = eb ? *eb : main_bufs();
    // G = conj(X) X^T  (NK x NK, column-major, Hermitian: lower triangle computed, upper mirrored)
    prof_sub = P_GEMM_GRAM;
    mpdo_status st = gemm_(NK, NK, (int)L, Xb, v2(sx, 0, 0, L, 0, 0, 1, 1), Yg ? Yg : Xb,
                           v2(Yg ? sY : sx, 0, 0, 1, 0, 0, L, 0), b.F, col_major(NK, b.sF), -1, 1);
    prof_sub = -1;
    if (st) return st;
    prof_start(P_OTHER, 0);
    CK(herm_fill_upper<R>(stream, B, NK, b.F, b.sF));
    prof_stop();
    ++launches;
    st = eig_(NK, kap, 1, &b);
    if (st) return st;
    // A[(s, nu, r)] = sum_nk V[nk, nu] X[nk][s][r]
    return gemm_(kap, (int)L, NK, b.U, v2(b.sU, 0, 0, NK, 0, 0, 1), Xb, row_major(L, sx), slot_ptr(out_slot),
                 v2(slot_elems, 0, 0, dr, dr, (int64_t)kap * dr, 1));
  }

  // ---------------------------------------------------------------- noisy gates
  mpdo_status apply(int nq, int q, const double* Uhost, const double* Udev, const mpdo_chanset* ch,
                    const int* idx_dev) override {
    if (q < 0 || q + nq > n) return MPDO_EINVAL;
    if (!ch || ch->nq != nq || ch->rpad > (nq == 3 ? 64 : RMAX)) return MPDO_EINVAL;
    if (!idx_dev && ch->count != 1 && ch->count != B) return MPDO_EINVAL;
    // a two-site split needs the centre on q or q + 1 (canonical environments on both sides); the other
    // site of the pair may be the non-isometric neighbour
    bool env = false;
    mpdo_status st = MPDO_OK;
    if (nq == 3) {
      st = check3(q, ch->rpad);
      if (!st) st = move_centre(q);
    } else if (nq == 2) {
      bool in_pair = (centre == q || centre == q + 1) && (dirty < 0 || dirty == q || dirty == q + 1);
      if (!in_pair) st = move_centre(q);
    } else if (centre != q || dirty >= 0) {
      // a 1q truncation needs every other site isometric: with the centre on q a non-isometric
      // neighbour is absorbed first (move_centre hops onto it and back)
      env = neighbour_trunc && (q == centre + 1 || q == centre - 1) && (dirty < 0 || dirty == q);
      if (!env) st = move_centre(q);
    }
    if (st) return st;
    // with one channel per chain and no index array, chain b uses channel b
    const int* idx = idx_dev;
    if (!idx && ch->count == B && B > 1) idx = iota;
    st = fuse_(nq, Uhost, Udev, ch, idx);
    if (st) return st;
    if (nq == 3) {
      st = apply3(q, ch->rpad);
      dirty = -1;
    } else if (nq == 2) {
      st = trunc_order == MPDO_TRUNC_KRAUS_FIRST ? apply2_kraus_first(q, ch->rpad) : apply2(q, ch->rpad);
      dirty = -1;
    } else {
      st = env ? apply1_neighbour(q, ch->rpad) : apply1(q, ch->rpad);
    }
    if (st) return st;
    return renorm_(nq == 1 ? q : centre);
  }

  // Nothing is renormalised (every readout but TRACE divides by Tr rho), so the state's norm decays
  // with each truncation's discarded weight; in complex64 storage a long lossy circuit would leave the
  // FP32 exponent range.  After every update the touched site is kept near unit scale by an exact
  // power of two, accumulated per chain in dExp2 and applied to the TRACE readout.
  mpdo_status renorm_(int q) {
    const int64_t elems = (int64_t)bond[q] * 2 * kraus[q] * bond[q + 1];
    prof_start(P_OTHER, 0);
    CK(renorm_sites<R>(stream, B, elems, site_ptr(q), slot_elems, dExp2));
    prof_stop();
    ++launches;
    return MPDO_OK;
  }

  // Noisy 1q gate (Fig. 2c) and the Kraus-leg truncation of its site (Eq. svdNoise) without forming
  // the extended site A' = (Khat (x) I) A, whose Kraus leg is r_k times wider.  The Gram of A' over
  // (l, p', r) follows from the Gram of A over its bonds,
  //   H[(p, n), (p'', n')] = sum_{l, r} conj(A[l, p, n, r]) Benv[l, p'', n', r],
  // as G = sum_{p, p''} (Khat_k^H Khat_k')[p, p''] H (kraus_gram); its top-kappa eigenvectors V are
  // folded into the gate, W = sum_k Khat_k V_k (kraus_fold), and the new site is one product
  // A'' = W A.  Benv is A itself with the centre on q, or A through the centre's environment when q is
  // its neighbour.  The site is read twice and only the truncated site is written.
  mpdo_status apply1_fold(int q, int rk, const C* Benv, int64_t bstride) {
    const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
    const int NK = rk * dn, NH = 2 * dn;
    const int64_t ld = (int64_t)2 * dn * dr;  // stride of l in a site
    const double site_bytes = (double)sizeof(C) * dl * ld * B;
    prof_sub = P_ONEQ;
    prof_bytes = site_bytes;  // the site streamed once (algorithmically)
    mpdo_status st = gemm_(NH, NH, dl * dr, site_ptr(q), v2(slot_elems, 0, 0, dr, dr, ld, 1, 1), Benv,
                           v2(bstride, dr, ld, 1, 0, 0, dr), wHk, row_major(NH, sHk));
    prof_sub = -1;
    prof_bytes = 0;
    if (st) return st;
    prof_start(P_OTHER, 8.0 * NK * NK * 12 * B);
    CK(kraus_gram<R>(stream, B, 2, rk, dn, wK, wHk, sHk, wF, sF));
    prof_stop();
    ++launches;
    const int kap = imin(kappa_max, imin(2 * dl * dr, NK));
    st = eig_(NK, kap, 1);
    if (st) return st;
    // W[(p', nu), (p, n)] = sum_k Khat_k[p', p] V[(k, n), nu]  (wHk, row-major 2 kap x 2 dn)
    prof_start(P_OTHER, 8.0 * 4 * kap * dn * rk * B);
    CK(kraus_fold<R>(stream, B, 2, rk, dn, kap, wK, wU, sU, NK, wHk, sHk));
    prof_stop();
    ++launches;
    // A''[l][(p', nu)][r] = sum_{(p, n)} W[(p', nu), (p, n)] A[l][(p, n)][r]
    const int so = take_slot();
    prof_sub = P_ONEQ;
    prof_bytes = site_bytes * (1.0 + (double)kap / dn);  // the site read again, the new site written
    st = gemm_(2 * kap, dl * dr, NH, wHk, row_major(NH, sHk), site_ptr(q), v2(slot_elems, 0, 0, dr, dr, ld, 1),
               slot_ptr(so), v2(slot_elems, 0, 0, dr, dr, (int64_t)2 * kap * dr, 1));
    prof_sub = -1;
    prof_bytes = 0;
    if (st) return st;
    give_slot(site_slot[q]);
    site_slot[q] = so;
    kraus[q] = kap;
    return MPDO_OK;
  }

  // Noisy 1q gate on a neighbour s of the centre c without moving the centre.  The Kraus-leg Gram of
  // s is its exact ancilla density: with every other site isometric, the sites beyond s contribute an
  // identity and the centre contributes its Gram over the shared bond, L (s = c + 1) or E (s = c - 1).
  // The kept subspace is therefore the one a centre move would have produced.
  mpdo_status apply1_neighbour(int q, int rk) {
    const int c = centre;
    const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
    const int64_t ld = (int64_t)2 * dn * dr;
    const C* Ac = site_ptr(c);
    mpdo_status st;
    if (q == c + 1) {
      // L[b, b'] = sum_(l,p,n) conj(Ac[(lpn), b]) Ac[(lpn), b'],  b over bond q (= dl)
      const int K = bond[c] * 2 * kraus[c];
      st = gemm_(dl, dl, K, Ac, v2(slot_elems, 0, 0, 1, 0, 0, dl, 1), Ac, row_major(dl, slot_elems), wE,
                 row_major(dl, sE));
      if (st) return st;
      // Benv[l][(p n r)] = sum_l' L[l, l'] A[l'][(p n r)]
      st = gemm_(dl, (int)ld, dl, wE, row_major(dl, sE), site_ptr(q), row_major(ld, slot_elems), wX, row_major(ld, sX));
    } else {
      // E[b, b'] = sum_(p,n,r) conj(Ac[b, (pnr)]) Ac[b', (pnr)],  b over bond c (= dr)
      const int K = 2 * kraus[c] * bond[c + 1];
      st = gemm_(dr, dr, K, Ac, v2(slot_elems, 0, 0, K, 0, 0, 1, 1), Ac, v2(slot_elems, 0, 0, 1, 0, 0, K), wE,
                 row_major(dr, sE));
      if (st) return st;
      // Benv[(l p n)][b] = sum_b' A[(l p n)][b'] E[b, b']
      st = gemm_(dl * 2 * dn, dr, dr, site_ptr(q), row_major(dr, slot_elems), wE, v2(sE, 0, 0, 1, 0, 0, dr), wX,
                 row_major(dr, sX));
    }
    if (st) return st;
    st = apply1_fold(q, rk, wX, sX);
    if (st) return st;
    dirty = q;
    return MPDO_OK;
  }
  int* iota = nullptr;  // device [0, 1, ..., B-1]
  int* dExp2 = nullptr;  // per chain: the represented state is the stored one times 2^dExp2

  mpdo_status apply1(int q, int rk) { return apply1_fold(q, rk, site_ptr(q), slot_elems); }

  mpdo_status apply2(int q, int rk) {
    const int dl = bond[q], dm = bond[q + 1], dr = bond[q + 2];
    const int dn1 = kraus[q], dn2 = kraus[q + 1];
    const int C2 = 2 * dm;
    // 1. QR of A1 as ((l, n1), (p1, b)) -> Q1 (m x x, wQ), R1 (x x 2dm, wQR), column-major ld m
    const int m = dl * dn1, x = imin(m, C2);
    QrArgs<R> qa;
    qa.m = m;
    qa.n = C2;
    qa.in = site_ptr(q);
    qa.vin = v2(slot_elems, dn1, (int64_t)2 * dn1 * dm, dm, dm, (int64_t)dn1 * dm, 1);
    qa.W = wQR;
    qa.wstride = sQR;
    qa.Qw = wQ;
    qa.qstride = sQR;
    qa.qout = nullptr;
    prof_start(P_QR, qr_flops(qa.m, qa.n) * B);
    CK(qr<R>(stream, B, qa));
    prof_stop();
    ++launches;
    const View R1 = col_major(m, sQR);
    // 2. E = A2 A2^H with A2 as (2dm) x (dn2 dr)
    const int K2 = dn2 * dr;
    mpdo_status st = gemm_(C2, C2, K2, site_ptr(q + 1), row_major(K2, slot_elems), site_ptr(q + 1),
                           v2(slot_elems, 0, 0, 1, 0, 0, K2, 1), wE, row_major(C2, sE));
    if (st) return st;
    // 3. T[c][a][c'][b] from E and the reduced superoperator of the fused gate
    prof_start(P_OTHER, 8.0 * 4 * 16 * dm * dm * B);
    CK(build_T<R>(stream, B, dm, wRt, wE, sE, wT, sT));
    prof_stop();
    ++launches;
    // 4. Z[x][(a, c', b)] = sum_c R1[x, c] T[c][(a, c', b)]
    const int NZ = 4 * C2;
    st = gemm_(x, NZ, C2, wQR, R1, wT, row_major(NZ, sT), wZ, row_major(NZ, sZ));
    if (st) return st;
    // 5. F'[(x, a), (x', b)] = sum_c' Z[(x, a), (c', b)] conj(R1[x', c']); batch index = b * B + chain
    {
      const int X2 = 2 * x;
      View va = v2(0, 0, 0, 2 * C2, 0, 0, 2);
      va.bdiv = B;
      va.bhi = 1;
      va.blo = sZ;
      View vb = v2(0, 0, 0, m, 0, 0, 1, 1);
      vb.bdiv = B;
      vb.bhi = 0;
      vb.blo = sQR;
      View vc = v2(0, 0, 0, 1, 0, 0, (int64_t)2 * X2);
      vc.bdiv = B;
      vc.bhi = X2;
      vc.blo = sF;
      st = gemm_(X2, x, C2, wZ, va, wQR, vb, wF, vc, 2 * B);
      if (st) return st;
    }
    // 6. bond: top kchi eigenpairs of F'
    const int kchi = imin(chi_max, imin(2 * x, 2 * dn2 * rk * dr));
    st = eig_(2 * x, kchi, 0);
    if (st) return st;
    // 7. A1' [l][p1'][n1][b'] = sum_x Q1[(l, n1), x] U[(x, p1'), b']
    const int s1 = take_slot();
    st = gemm_(m, 2 * kchi, x, wQ, col_major(m, sQR), wU, v2(sU, 0, 0, 2, kchi, 1, (int64_t)2 * x),
               slot_ptr(s1), v2(slot_elems, dn1, (int64_t)2 * dn1 * kchi, kchi, kchi, (int64_t)dn1 * kchi, 1));
    if (st) return st;
    // 8. H[(b', p1')][(p1, bb)] = sum_x conj(U[(x, p1'), b']) R1[x, (p1, bb)]
    st = gemm_(2 * kchi, C2, x, wU, v2(sU, 2, (int64_t)2 * x, 1, 0, 0, 2, 1), wQR, R1, wH, row_major(C2, sH));
    if (st) return st;
    // 9. Y[(b', p2', k)][(bb, p2)] = sum Khat_k[(p1' p2'), (p1 p2)] H[(b', p1')][(p1, bb)]
    prof_start(P_OTHER, 8.0 * 4 * kchi * 2 * rk * C2 * B);
    CK(build_Y<R>(stream, B, kchi, dm, rk, wK, wH, sH, wY, sY));
    prof_stop();
    ++launches;
    // 10. X (Kraus-major [(k, n2)][(b', p2')][r]) = Y . A2
    const int S = 2 * kchi, NK = rk * dn2;
    const int64_t Lx = (int64_t)S * dr;
    prof_sub = P_GEMM_X;
    st = gemm_(S * rk, K2, C2, wY, row_major(C2, sY), site_ptr(q + 1), row_major(K2, slot_elems), wX,
               v2(sX, rk, dr, (int64_t)dn2 * Lx, dr, Lx, 1));
    prof_sub = -1;
    if (st) return st;
    // 11-13. Kraus-leg truncation of site q+1
    const int kap = imin(kappa_max, imin((int)Lx, NK));
    const int s2 = take_slot();
    st = kappa_truncate_X(NK, S, dr, kap, s2);
    if (st) return st;
    give_slot(site_slot[q]);
    give_slot(site_slot[q + 1]);
    site_slot[q] = s1;
    site_slot[q + 1] = s2;
    bond[q + 1] = kchi;
    kraus[q + 1] = kap;
    centre = q + 1;
    return MPDO_OK;
  }

  // Two-qubit update in the Kraus-first order: the merged tensor's new Kraus leg (k, n2) is truncated to
  // kappa_max (Eq. svdNoise) before the bond split (Fig. 3b).  Theta is never formed: with
  // Theta0 = R1 A2 (the pair reduced by the QR of A1), the leg's Gram is assembled from the small Gram
  // H of Theta0 over (x, r) and the fused gate, the kept directions are folded into the gate
  // (W = sum_k Khat_k V_k), and Theta' = W Theta0 carries kappa instead of r_k kappa Kraus indices
  // into the split.  The centre ends on q + 1.
  mpdo_status apply2_kraus_first(int q, int rk) {
    const int dl = bond[q], dm = bond[q + 1], dr = bond[q + 2];
    const int dn1 = kraus[q], dn2 = kraus[q + 1];
    const int C2 = 2 * dm;
    // 1. QR of A1 as ((l, n1), (p1, b)) -> Q1 (m x x, wQ), R1 (x x 2dm, wQR), column-major ld m
    const int m = dl * dn1, x = imin(m, C2);
    QrArgs<R> qa;
    qa.m = m;
    qa.n = C2;
    qa.in = site_ptr(q);
    qa.vin = v2(slot_elems, dn1, (int64_t)2 * dn1 * dm, dm, dm, (int64_t)dn1 * dm, 1);
    qa.W = wQR;
    qa.wstride = sQR;
    qa.Qw = wQ;
    qa.qstride = sQR;
    qa.qout = nullptr;
    prof_start(P_QR, qr_flops(qa.m, qa.n) * B);
    CK(qr<R>(stream, B, qa));
    prof_stop();
    ++launches;
    // 2. Theta0[(x, p1)][(p2, n2, r)] = sum_bb R1[x, (p1, bb)] A2[bb][(p2, n2, r)]  (wX)
    const int N0 = 2 * dn2 * dr;
    mpdo_status st = gemm_(2 * x, N0, dm, wQR, v2(sQR, 2, 1, (int64_t)dm * m, 0, 0, m), site_ptr(q + 1),
                           row_major(N0, slot_elems), wX, row_major(N0, sX));
    if (st) return st;
    // 3. H[(p, n2), (p'', n2')] = sum_{x, r} conj(Theta0[x, p, n2, r]) Theta0[x, p'', n2', r]  (wHk, row-major)
    const int NH = 4 * dn2;
    const int64_t ld0 = (int64_t)4 * dn2 * dr;  // stride of x in Theta0
    st = gemm_(NH, NH, x * dr, wX, v2(sX, 0, 0, dr, dr, ld0, 1, 1), wX, v2(sX, dr, ld0, 1, 0, 0, dr), wHk,
               row_major(NH, sHk));
    if (st) return st;
    // 4. the Kraus-leg Gram G (rk dn2 square, column-major, wF) and its top-kappa eigenpairs
    const int NK = rk * dn2;
    prof_start(P_OTHER, 8.0 * NK * NK * 80 * B);
    CK(kraus_gram<R>(stream, B, 4, rk, dn2, wK, wHk, sHk, wF, sF));
    prof_stop();
    ++launches;
    const int kap = imin(kappa_max, imin(NK, x * 4 * dr));
    st = eig_(NK, kap, 1);
    if (st) return st;
    // 5. W[(p', nu), (p, n2)] = sum_k Khat_k[p', p] V[(k, n2), nu]  (wHk, row-major 4 kap x 4 dn2)
    prof_start(P_OTHER, 8.0 * 16 * kap * dn2 * rk * B);
    CK(kraus_fold<R>(stream, B, 4, rk, dn2, kap, wK, wU, sU, NK, wHk, sHk));
    prof_stop();
    ++launches;
    // 6. Theta'[x][(p1', p2')][nu][r] = sum_{(p, n2)} W[(p', nu), (p, n2)] Theta0[x][(p, n2)][r]  (wY)
    st = gemm_(4 * kap, x * dr, NH, wHk, row_major(NH, sHk), wX, v2(sX, 0, 0, dr, dr, ld0, 1), wY,
               v2(sY, 0, 0, dr, dr, (int64_t)4 * kap * dr, 1));
    if (st) return st;
    // 7. F[(x, p1'), (x', p1'')] = sum_{(p2', nu, r)} Theta' conj(Theta')  (wF, column-major, Hermitian)
    const int NF = 2 * x, KF = 2 * kap * dr;
    st = gemm_(NF, NF, KF, wY, row_major(KF, sY), wY, v2(sY, 0, 0, 1, 0, 0, KF, 1), wF, col_major(NF, sF), -1, 1);
    if (st) return st;
    prof_start(P_OTHER, 0);
    CK(herm_fill_upper<R>(stream, B, NF, wF, sF));
    prof_stop();
    ++launches;
    // 8. bond: top kchi eigenpairs of F
    const int kchi = imin(chi_max, imin(NF, KF));
    st = eig_(NF, kchi, 0);
    if (st) return st;
    // 9. A1' [l][p1'][n1][b'] = sum_x Q1[(l, n1), x] U[(x, p1'), b']
    const int s1 = take_slot();
    st = gemm_(m, 2 * kchi, x, wQ, col_major(m, sQR), wU, v2(sU, 0, 0, 2, kchi, 1, (int64_t)2 * x),
               slot_ptr(s1), v2(slot_elems, dn1, (int64_t)2 * dn1 * kchi, kchi, kchi, (int64_t)dn1 * kchi, 1));
    if (st) return st;
    // 10. A2'[b'][(p2', nu, r)] = sum_{(x, p1')} conj(U[(x, p1'), b']) Theta'[(x, p1'), (p2', nu, r)]
    const int s2 = take_slot();
    st = gemm_(kchi, KF, NF, wU, v2(sU, 0, 0, NF, 0, 0, 1, 1), wY, row_major(KF, sY), slot_ptr(s2),
               row_major(KF, slot_elems));
    if (st) return st;
    give_slot(site_slot[q]);
    give_slot(site_slot[q + 1]);
    site_slot[q] = s1;
    site_slot[q + 1] = s2;
    bond[q + 1] = kchi;
    kraus[q + 1] = kap;
    centre = q + 1;
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- three-site update
  // Workspace of the three-site update, sized from the caps at the first three-qubit gate: the
  // merged tensor with the new Kraus leg is up to 2x * 2dn2 * rk * dn3 * 2dr <= 1024 chi^2 kappa^2
  // elements per chain (x <= 2 chi, rk <= 64).
  mpdo_status alloc3() {
    if (w3a) return MPDO_OK;
    if (capturing) return MPDO_ESTATE;
    const int64_t X = chi_max, K = kappa_max;
    const int n3 = (int)lmax(2 * X * K, 64 * K);  // <= 512 (check3)
    s3a = 512 * K * K * X * X;
    s3b = lmax(16 * K * K * X * X, 128 * K * X * X);
    s3c = 1024 * K * K * X * X;
    s3F = (int64_t)n3 * n3;
    s3Eval = n3 + 1;
    s3Scr = eig_scratch_elems(n3, n3);
    bool ok = dmalloc(&w3a, s3a * B) == cudaSuccess && dmalloc(&w3b, s3b * B) == cudaSuccess &&
              dmalloc(&w3c, s3c * B) == cudaSuccess && dmalloc(&w3K, (int64_t)64 * 64 * B) == cudaSuccess &&
              dmalloc(&w3F, s3F * B) == cudaSuccess && dmalloc(&w3U, s3F * B) == cudaSuccess &&
              dmalloc(&w3Eval, s3Eval * B) == cudaSuccess && dmalloc(&w3Scr, s3Scr * B) == cudaSuccess;
    if (ok && !std::is_same<R, ER>::value)
      ok = dmalloc(&w3F64, s3F * B) == cudaSuccess && dmalloc(&w3U64, s3F * B) == cudaSuccess;
    if (!ok) {
      void* ptrs[] = {w3a, w3b, w3c, w3K, w3F, w3U, w3F64, w3U64, w3Eval, w3Scr};
      for (void* p : ptrs)
        if (p) cudaFree(p);
      w3a = w3b = w3c = w3K = w3F = w3U = nullptr;
      w3F64 = w3U64 = nullptr;
      w3Eval = w3Scr = nullptr;
      cudaGetLastError();
      return MPDO_ENOMEM;
    }
    return MPDO_OK;
  }
  // The shapes of a three-site update on (q, q+1, q+2) must fit the eigensolver (order <= 512) and
  // the workspace; checked before anything is launched.
  mpdo_status check3(int q, int rk) {
    if (q < 0 || q + 3 > n || rk < 1 || rk > 64) return MPDO_EINVAL;
    if (2 * chi_max * kappa_max > 512 || 64 * kappa_max > 512) return MPDO_EINVAL;
    mpdo_status st = alloc3();
    if (st) return st;
    const int dl = bond[q], d1 = bond[q + 1], d2 = bond[q + 2], dr = bond[q + 3];
    const int dn1 = kraus[q], dn2 = kraus[q + 1], dn3 = kraus[q + 2];
    const int x = imin(dl * dn1, 2 * d1);
    const int64_t C1 = (int64_t)4 * dn2 * rk * dn3 * dr;
    const int k1 = (int)std::min<int64_t>(chi_max, std::min<int64_t>(2 * x, C1));
    const int M2 = 2 * k1 * dn2, NK = rk * dn3;
    const int64_t Cc = (int64_t)rk * dn3 * 2 * dr;
    const int k2 = (int)std::min<int64_t>(chi_max, std::min<int64_t>(M2, Cc));
    if (2 * x > 512 || M2 > 512 || NK > 512) return MPDO_EINVAL;
    if ((int64_t)2 * x * 2 * dn2 * d2 > s3a || (int64_t)k1 * C1 > s3a || (int64_t)4 * x * dn2 * 2 * dn3 * dr > s3b ||
        (int64_t)NK * 2 * k2 * dr > s3b || (int64_t)2 * x * C1 > s3c || (int64_t)M2 * M2 > s3F ||
        (int64_t)NK * NK > s3F || (int64_t)4 * x * x > sF)
      return MPDO_EINVAL;
    return MPDO_OK;
  }
  // Noisy three-qubit channel on (q, q+1, q+2), e.g. the crosstalk channel from a tomography of a
  // two-qubit gate with its neighbour (Fig. 13b), with the new Kraus leg on site q+2 and the centre on
  // q: the pair reduced by the QR of A1 (Q1 R1), Theta0 = R1 A2 A3, the gate applied (gate3), the bond
  // (q, q+1) split by the top-chi eigenvectors U1 of F1 = Theta Theta^H over (x, p1'), the rest
  // R = U1^H Theta split at (q+1, q+2) by the top-chi eigenvectors U2 of F2 = R R^H over (b1, p2', n2),
  // and site q+2's Kraus leg truncated (Eq. svdNoise).  The centre ends on q + 2.
  mpdo_status apply3(int q, int rk) {
    const int dl = bond[q], d1 = bond[q + 1], d2 = bond[q + 2], dr = bond[q + 3];
    const int dn1 = kraus[q], dn2 = kraus[q + 1], dn3 = kraus[q + 2];
    const int C2 = 2 * d1, m = dl * dn1, x = imin(m, C2);
    // 1. QR of A1 as ((l, n1), (p1, b)) -> Q1 (m x x, wQ), R1 (x x 2 d1, wQR), column-major ld m
    QrArgs<R> qa;
    qa.m = m;
    qa.n = C2;
    qa.in = site_ptr(q);
    qa.vin = v2(slot_elems, dn1, (int64_t)2 * dn1 * d1, d1, d1, (int64_t)dn1 * d1, 1);
    qa.W = wQR;
    qa.wstride = sQR;
    qa.Qw = wQ;
    qa.qstride = sQR;
    qa.qout = nullptr;
    prof_start(P_QR, qr_flops(qa.m, qa.n) * B);
    CK(qr<R>(stream, B, qa));
    prof_stop();
    ++launches;
    // 2. T12[(x, p1)][(p2, n2, b2)] = sum_b R1[x, (p1, b)] A2[b][(p2, n2, b2)]  (w3a)
    const int N12 = 2 * dn2 * d2;
    mpdo_status st = gemm_(2 * x, N12, d1, wQR, v2(sQR, 2, 1, (int64_t)d1 * m, 0, 0, m), site_ptr(q + 1),
                           row_major(N12, slot_elems), w3a, row_major(N12, s3a));
    if (st) return st;
    // 3. Theta0[(x, p1, p2, n2)][(p3, n3, r)] = sum_b2 T12[(x, p1, p2, n2), b2] A3[b2][(p3, n3, r)]  (w3b)
    const int N3 = 2 * dn3 * dr;
    st = gemm_(4 * x * dn2, N3, d2, w3a, row_major(d2, s3a), site_ptr(q + 2), row_major(N3, slot_elems), w3b,
               row_major(N3, s3b));
    if (st) return st;
    // 4. Theta[(x, p1')][(p2', n2, k, n3, p3', r)]  (w3c)
    const int64_t C1 = (int64_t)4 * dn2 * rk * dn3 * dr;
    prof_start(P_OTHER, 8.0 * 8 * 2 * x * C1 * B);
    CK(gate3<R>(stream, B, x, dn2, dn3, dr, rk, w3K, w3b, s3b, w3c, s3c));
    prof_stop();
    ++launches;
    // 5. bond (q, q+1): F1 = Theta Theta^H over (x, p1') (wF, column-major), its top k1 eigenpairs
    const int X2 = 2 * x;
    st = gemm_(X2, X2, (int)C1, w3c, row_major(C1, s3c), w3c, v2(s3c, 0, 0, 1, 0, 0, C1, 1), wF, col_major(X2, sF),
               -1, 1);
    if (st) return st;
    prof_start(P_OTHER, 0);
    CK(herm_fill_upper<R>(stream, B, X2, wF, sF));
    prof_stop();
    ++launches;
    const int k1 = (int)std::min<int64_t>(chi_max, std::min<int64_t>(X2, C1));
    st = eig_(X2, k1, 0);
    if (st) return st;
    // 6. A1' [l][p1'][n1][b'] = sum_x Q1[(l, n1), x] U1[(x, p1'), b']
    const int s1 = take_slot();
    st = gemm_(m, 2 * k1, x, wQ, col_major(m, sQR), wU, v2(sU, 0, 0, 2, k1, 1, (int64_t)X2), slot_ptr(s1),
               v2(slot_elems, dn1, (int64_t)2 * dn1 * k1, k1, k1, (int64_t)dn1 * k1, 1));
    if (st) return st;
    // 7. R[b1][(p2', n2, k, n3, p3', r)] = sum_i conj(U1[i, b1]) Theta[i][...]  (w3a)
    st = gemm_(k1, (int)C1, X2, wU, v2(sU, 0, 0, X2, 0, 0, 1, 1), w3c, row_major(C1, s3c), w3a, row_major(C1, s3a));
    if (st) return st;
    // 8. bond (q+1, q+2): F2 = R R^H over (b1, p2', n2) (w3F), its top k2 eigenpairs U2 (w3U)
    const int M2 = 2 * k1 * dn2;
    const int64_t Cc = (int64_t)rk * dn3 * 2 * dr;
    st = gemm_(M2, M2, (int)Cc, w3a, row_major(Cc, s3a), w3a, v2(s3a, 0, 0, 1, 0, 0, Cc, 1), w3F,
               col_major(M2, s3F), -1, 1);
    if (st) return st;
    prof_start(P_OTHER, 0);
    CK(herm_fill_upper<R>(stream, B, M2, w3F, s3F));
    prof_stop();
    ++launches;
    const EigBufs b3 = {w3F, w3U, s3F, s3F, w3F64, w3U64, w3Eval, w3Scr, s3Eval, s3Scr};
    const int k2 = (int)std::min<int64_t>(chi_max, std::min<int64_t>(M2, Cc));
    st = eig_(M2, k2, 0, &b3);
    if (st) return st;
    // 9. A2' [b1][p2'][n2][b2] = U2[(b1, p2', n2), b2]
    const int s2 = take_slot();
    CK(copy_view<R>(stream, B, M2, k2, w3U, col_major(M2, s3F), slot_ptr(s2), row_major(k2, slot_elems)));
    ++launches;
    // 10. X[(k, n3)][(b2, p3')][r] = sum_i conj(U2[i, b2]) R[i][(k, n3, p3', r)]  (w3b, Kraus-major)
    st = gemm_(k2, (int)Cc, M2, w3U, v2(s3F, 0, 0, M2, 0, 0, 1, 1), w3a, row_major(Cc, s3a), w3b,
               v2(s3b, 0, 0, 2 * dr, 2 * dr, (int64_t)2 * k2 * dr, 1));
    if (st) return st;
    // 11. Kraus-leg truncation of site q+2
    const int NK = rk * dn3;
    const int kap = imin(kappa_max, imin(2 * k2 * dr, NK));
    const int s3 = take_slot();
    st = kappa_truncate_X(NK, 2 * k2, dr, kap, s3, nullptr, w3b, s3b, &b3);
    if (st) return st;
    give_slot(site_slot[q]);
    give_slot(site_slot[q + 1]);
    give_slot(site_slot[q + 2]);
    site_slot[q] = s1;
    site_slot[q + 1] = s2;
    site_slot[q + 2] = s3;
    bond[q + 1] = k1;
    bond[q + 2] = k2;
    kraus[q + 2] = kap;
    centre = q + 2;
    return MPDO_OK;
  }

  mpdo_status truncate(int q, int kappa, double* disc) override {
    if (q < 0 || q >= n) return MPDO_EINVAL;
    mpdo_status st = move_centre(q);
    if (st) return st;
    const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
    int kap = kappa > 0 ? kappa : kappa_max;
    kap = imin(kap, imin(dn, 2 * dl * dr));
    std::vector<double> before;
    if (disc) {
      before.resize(3 * (size_t)B);
      CK(cudaMemcpyAsync(before.data(), dDisc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, stream));
    }
    // site [l][p][n][r] -> Kraus-major X[n][(l, p)][r]
    const int S = 2 * dl;
    CK(copy_view<R>(stream, B, dn, S * dr, site_ptr(q), v2(slot_elems, 0, 0, dr, dr, (int64_t)dn * dr, 1), wX,
                    row_major((int64_t)S * dr, sX)));
    ++launches;
    const int so = take_slot();
    st = kappa_truncate_X(dn, S, dr, kap, so);
    if (st) return st;
    give_slot(site_slot[q]);
    site_slot[q] = so;
    kraus[q] = kap;
    if ((st = renorm_(q))) return st;
    if (disc) {
      std::vector<double> after(3 * (size_t)B);
      CK(cudaMemcpyAsync(after.data(), dDisc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      for (int b = 0; b < B; ++b) disc[b] = after[3 * b + 1] - before[3 * b + 1];
    }
    return MPDO_OK;
  }

  // Global bond truncation of Sec. II.D (Fig. 3b): the centre is moved to the last site by QR
  // decompositions from left to right (canonical form), then each bond (c-1, c) is truncated to chi
  // from right to left.  With the centre on c, the Gram G = T_c T_c^H over the left bond (T_c as an
  // l x (p, n, r) matrix) has the squared Schmidt values of the bond as eigenvalues; with U its top
  // chi eigenvectors, T_c <- U^H T_c and T_{c-1} <- T_{c-1} U project the bond onto the kept
  // Schmidt directions, and an LQ step moves the centre on to c-1.  The centre ends on site 0.
  mpdo_status truncate_bonds(int chi, double* disc) override {
    if (chi < 1) return MPDO_EINVAL;
    std::vector<double> before;
    if (disc) {
      before.resize(3 * (size_t)B);
      CK(cudaMemcpyAsync(before.data(), dDisc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, stream));
    }
    mpdo_status st = move_centre(n - 1);
    if (st) return st;
    for (int c = n - 1; c >= 1; --c) {
      const int dl = bond[c], dn = kraus[c], dr = bond[c + 1];
      const int L = 2 * dn * dr;
      const int k = imin(chi, imin(dl, L));
      if (k < dl) {
        // G[l, l'] = sum_j T_c[l, j] conj(T_c[l', j]), column-major Hermitian (wF)
        st = gemm_(dl, dl, L, site_ptr(c), row_major(L, slot_elems), site_ptr(c), v2(slot_elems, 0, 0, 1, 0, 0, L, 1),
                   wF, col_major(dl, sF), -1, 1);
        if (st) return st;
        prof_start(P_OTHER, 0);
        CK(herm_fill_upper<R>(stream, B, dl, wF, sF));
        prof_stop();
        ++launches;
        st = eig_(dl, k, 0);
        if (st) return st;
        // T_c' [i][j] = sum_l conj(U[l, i]) T_c[l][j]
        const int sa = take_slot();
        st = gemm_(k, L, dl, wU, v2(sU, 0, 0, dl, 0, 0, 1, 1), site_ptr(c), row_major(L, slot_elems), slot_ptr(sa),
                   row_major(L, slot_elems));
        if (st) return st;
        // T_{c-1}' [(l, p, n)][i] = sum_b T_{c-1}[(l, p, n)][b] U[b, i]
        const int M = bond[c - 1] * 2 * kraus[c - 1];
        const int sb = take_slot();
        st = gemm_(M, k, dl, site_ptr(c - 1), row_major(dl, slot_elems), wU, col_major(dl, sU), slot_ptr(sb),
                   row_major(k, slot_elems));
        if (st) return st;
        give_slot(site_slot[c]);
        give_slot(site_slot[c - 1]);
        site_slot[c] = sa;
        site_slot[c - 1] = sb;
        bond[c] = k;
      }
      st = shift_left(c);
      if (st) return st;
      centre = c - 1;
    }
    if ((st = renorm_(0))) return st;
    if (disc) {
      std::vector<double> after(3 * (size_t)B);
      CK(cudaMemcpyAsync(after.data(), dDisc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      for (int b = 0; b < B; ++b) disc[b] = after[3 * b] - before[3 * b];
    }
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- readouts
  C* envl(int q) { return envL + (int64_t)q * B * sEnv; }
  C* envr(int q) { return envR + (int64_t)q * B * sEnv; }

  // E' = transfer of E (dl x dl) through site q, Z on the physical index when z
  mpdo_status left_step(int q, const C* E, C* out, bool z) {
    const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
    const int N = 2 * dn * dr;
    // tmp[l'][(p, n, r)] = sum_l E[l, l'] conj(A[l, (p, n, r)])
    mpdo_status st = gemm_(dl, N, dl, E, v2(sEnv, 0, 0, 1, 0, 0, dl), site_ptr(q), v2(slot_elems, 0, 0, N, 0, 0, 1, 1),
                           tmpA, row_major(N, sTmp));
    if (st) return st;
    if (z) {
      CK(scale_odd<R>(stream, B, (int64_t)dl * N, (int64_t)dn * dr, R(-1), tmpA, sTmp));
      ++launches;
    }
    // out[r, r'] = sum_{(l', p, n)} tmp[(l', p, n), r] A[(l', p, n), r']
    return gemm_(dr, dr, dl * 2 * dn, tmpA, v2(sTmp, 0, 0, 1, 0, 0, dr), site_ptr(q), row_major(dr, slot_elems), out,
                 row_major(dr, sEnv));
  }
  // E = right transfer of Rr (dr x dr) through site q
  mpdo_status right_step(int q, const C* Rr, C* out, bool z) {
    const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
    const int M = dl * 2 * dn;
    mpdo_status st = gemm_(M, dr, dr, site_ptr(q), row_major(dr, slot_elems), Rr, v2(sEnv, 0, 0, 1, 0, 0, dr), tmpA,
                           row_major(dr, sTmp));
    if (st) return st;
    if (z) {
      CK(scale_odd<R>(stream, B, (int64_t)M * dr, (int64_t)dn * dr, R(-1), tmpA, sTmp));
      ++launches;
    }
    const int K = 2 * dn * dr;
    return gemm_(dl, dl, K, site_ptr(q), v2(slot_elems, 0, 0, K, 0, 0, 1, 1), tmpA, v2(sTmp, 0, 0, 1, 0, 0, K), out,
                 row_major(dl, sEnv));
  }
  mpdo_status one_env(C* E) {
    cplx<R> one = mk<R>(1, 0);
    for (int b = 0; b < B; ++b) {
      CK(fill<R>(stream, 1, E + (int64_t)b * sEnv, one));
      ++launches;
    }
    return MPDO_OK;
  }
  // sum_{r r'} E[r, r'] Rr[r, r'] per chain (Rr Hermitian: = sum conj(Rr^T) E, done as a dot of E with Rr^T*)
  mpdo_status close_(const C* E, const C* Rr, int d, std::vector<double>& re) {
    // tmpB = conj(Rr), so that dot(tmpB, E) = sum E[r, r'] Rr[r, r']
    CK(copy_view<R>(stream, B, d, d, Rr, v2(sEnv, 0, 0, d, 0, 0, 1, 1), tmpB, row_major(d, sTmp)));
    ++launches;
    CK(dot_batch<R>(stream, B, (int64_t)d * d, tmpB, sTmp, E, sEnv, dDot));
    ++launches;
    std::vector<cplx<double>> h(B);
    CK(cudaMemcpyAsync(h.data(), dDot, sizeof(cplx<double>) * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    re.resize(B);
    for (int b = 0; b < B; ++b) re[b] = h[b].x;
    return MPDO_OK;
  }
  mpdo_status build_envs() {
    mpdo_status st = one_env(envl(0));
    if (st) return st;
    for (int q = 0; q < n; ++q)
      if ((st = left_step(q, envl(q), envl(q + 1), false))) return st;
    if ((st = one_env(envr(n)))) return st;
    for (int q = n - 1; q >= 0; --q)
      if ((st = right_step(q, envr(q + 1), envr(q), false))) return st;
    return MPDO_OK;
  }
  mpdo_status trace_(std::vector<double>& tr) { return close_(envl(n), envr(n), 1, tr); }

  mpdo_status zz_pairs(const std::vector<std::pair<int, int>>& pairs, std::vector<std::vector<double>>& vals) {
    vals.assign(pairs.size(), std::vector<double>(B, 0));
    // group by i
    for (int i = 0; i < n; ++i) {
      int jmax = -1;
      for (auto& p : pairs)
        if (p.first == i) jmax = p.second > jmax ? p.second : jmax;
      if (jmax < 0) continue;
      // ping-pong E through tmp env slots: use envL storage of a scratch index n? use two buffers in wE/wT
      C* Ea = wE;  // sE = 4 X^2 >= X^2
      C* Eb = wT;
      mpdo_status st = left_step_to(i, envl(i), Ea, true);
      if (st) return st;
      for (int j = i + 1; j <= jmax; ++j) {
        // value with Z at j
        if ((st = left_step_to(j, Ea, Eb, true))) return st;
        bool need = false;
        for (auto& p : pairs) need |= (p.first == i && p.second == j);
        if (need) {
          std::vector<double> v;
          if ((st = close_generic(Eb, envr(j + 1), bond[j + 1], v))) return st;
          for (size_t t = 0; t < pairs.size(); ++t)
            if (pairs[t].first == i && pairs[t].second == j) vals[t] = v;
        }
        if (j < jmax) {
          if ((st = left_step_to(j, Ea, Eb, false))) return st;
          std::swap(Ea, Eb);
        }
      }
    }
    return MPDO_OK;
  }
  // left_step writing into a workspace buffer with env stride (sE, sT >= sEnv are used with stride sEnv)
  mpdo_status left_step_to(int q, const C* E, C* out, bool z) { return left_step(q, E, out, z); }
  mpdo_status close_generic(const C* E, const C* Rr, int d, std::vector<double>& re) { return close_(E, Rr, d, re); }

  // <a| rho |b> element transfer for a, b in {0, 1} on every site
  mpdo_status element_(int a, int bsel, std::vector<double>& re, std::vector<double>& im) {
    return element_bits(std::vector<int>(n, a), std::vector<int>(n, bsel), re, im);
  }
  // <a| rho |b> for computational-basis strings a, b (one physical index per site)
  mpdo_status element_bits(const std::vector<int>& a, const std::vector<int>& bb, std::vector<double>& re,
                           std::vector<double>& im) {
    C* Ea = wE;
    C* Eb = wT;
    mpdo_status st = one_env(Ea);
    if (st) return st;
    for (int q = 0; q < n; ++q) {
      const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
      const int N = dn * dr;
      const C* A = site_ptr(q);
      // tmp[l'][(n, r)] = sum_l E[l, l'] A[l, a, n, r]
      st = gemm_(dl, N, dl, Ea, v2(sEnv, 0, 0, 1, 0, 0, dl), A + (int64_t)a[q] * N, v2(slot_elems, 0, 0, 2 * N, 0, 0, 1),
                 tmpA, row_major(N, sTmp));
      if (st) return st;
      // E'[r, r'] = sum_{(l', n)} tmp[(l', n), r] conj(A[l', b, n, r'])
      st = gemm_(dr, dr, dl * dn, tmpA, v2(sTmp, 0, 0, 1, 0, 0, dr), A + (int64_t)bb[q] * N,
                 v2(slot_elems, dn, (int64_t)2 * N, dr, 0, 0, 1, 1), Eb, row_major(dr, sEnv));
      if (st) return st;
      std::swap(Ea, Eb);
    }
    // element [0, 0] of every chain's environment gathered into one contiguous buffer, one copy
    std::vector<C> hc(B);
    CK(copy_view<R>(stream, B, 1, 1, Ea, v2(sEnv, 0, 0, 1, 0, 0, 1), tmpB, row_major(1, 1)));
    ++launches;
    CK(cudaMemcpyAsync(hc.data(), tmpB, sizeof(C) * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    re.resize(B);
    im.resize(B);
    for (int b = 0; b < B; ++b) {
      re[b] = (double)hc[b].x;
      im[b] = (double)hc[b].y;
    }
    return MPDO_OK;
  }

  // The whole bitstring distribution <z| rho |z> / Tr rho of every chain (Sec. IV.A, IV.C): the
  // element transfer of element_bits for all 2^q prefixes of a chain at once, prefixes as the batch
  // of the products, E_{(A, p)}[r, r'] = sum_{l, l', n} E_A[l, l'] T[l, p, n, r] conj(T[l', p, n, r']),
  // so the distribution costs 4 n batched products per chain instead of one sweep per bitstring.
  // out: B x 2^n, qubit 0 most significant; n <= 15.
  mpdo_status distribution(double* out) override {
    if (n > 15) return MPDO_EINVAL;
    mpdo_status st = clean();
    if (st) return st;
    int64_t eMax = 1, tMax = 1;
    for (int q = 0; q < n; ++q) {
      const int64_t P = (int64_t)1 << q;
      eMax = lmax(eMax, 2 * P * bond[q + 1] * bond[q + 1]);
      eMax = lmax(eMax, P * bond[q] * bond[q]);
      tMax = lmax(tMax, P * bond[q] * kraus[q] * bond[q + 1]);
    }
    C *E0 = nullptr, *E1 = nullptr, *Tm = nullptr;
    if (dmalloc(&E0, eMax) != cudaSuccess || dmalloc(&E1, eMax) != cudaSuccess || dmalloc(&Tm, tMax) != cudaSuccess) {
      if (E0) cudaFree(E0);
      if (E1) cudaFree(E1);
      cudaGetLastError();
      return MPDO_ENOMEM;
    }
    const int64_t Z = (int64_t)1 << n;
    std::vector<C> h((size_t)Z);
    for (int b = 0; b < B && !st; ++b) {
      C* Ea = E0;
      C* Eb = E1;
      CK(fill<R>(stream, 1, Ea, mk<R>(1, 0)));
      ++launches;
      for (int q = 0; q < n && !st; ++q) {
        const int dl = bond[q], dn = kraus[q], dr = bond[q + 1];
        const int N = dn * dr, P = 1 << q;
        const C* A = site_ptr(q) + (int64_t)b * slot_elems;
        for (int p = 0; p < 2 && !st; ++p) {
          // Tm[A][l'][(n, r)] = sum_l E_A[l, l'] T[l, p, n, r]
          View ve = v2((int64_t)dl * dl, 0, 0, 1, 0, 0, dl);
          View va = v2(0, 0, 0, 2 * N, 0, 0, 1);
          View vt = row_major(N, (int64_t)dl * N);
          st = gemm_(dl, N, dl, Ea, ve, A + (int64_t)p * N, va, Tm, vt, P);
          if (st) break;
          // E_{(A, p)}[r, r'] = sum_{(l', n)} Tm[A][(l', n), r] conj(T[l', p, n, r'])
          View vt2 = v2((int64_t)dl * N, 0, 0, 1, 0, 0, dr);
          View vb = v2(0, dn, (int64_t)2 * N, dr, 0, 0, 1, 1);
          View vo = row_major(dr, (int64_t)2 * dr * dr);
          st = gemm_(dr, dr, dl * dn, Tm, vt2, A + (int64_t)p * N, vb, Eb + (int64_t)p * dr * dr, vo, P);
        }
        std::swap(Ea, Eb);
      }
      if (st) break;
      CK(cudaMemcpyAsync(h.data(), Ea, sizeof(C) * Z, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      double tot = 0;
      for (int64_t z = 0; z < Z; ++z) tot += (double)h[(size_t)z].x;
      for (int64_t z = 0; z < Z; ++z) out[(size_t)b * Z + z] = tot > 0 ? (double)h[(size_t)z].x / tot : 0.0;
      if (!(tot > 0) || !std::isfinite(tot)) st = MPDO_ENOCONV;
    }
    cudaFree(E0);
    cudaFree(E1);
    cudaFree(Tm);
    return st;
  }

  // Tr rho^2 by the four-copy transfer (one chain at a time)
  // Tr rho^2 per chain: a left-to-right sweep of the four-copy environment E[a][b][c][d]
  // (ket, bra, ket, bra bond indices; D^4 elements) through four GEMMs per site, each about
  // 2 dn D^5 complex multiply-adds, with permutes between them.  The intermediates are processed in
  // chunks of the last environment index d (the partial results add up in the final GEMM), so
  // their size is bounded by a share of the free device memory; the buffers are kept for later calls.
  mpdo_status purity_(std::vector<double>& out) {
    const int64_t X = chi_max, K = kappa_max;
    // intermediate elements per unit of d-chunk at the caps
    auto per_d = [](int64_t D, int64_t dn, int64_t dr) {
      int64_t u1 = D * D * 2 * dn * dr, u2 = D * 4 * dr * dr, u3 = 2 * dn * dr * dr * dr;
      int64_t u = u1 > u2 ? u1 : u2;
      return u > u3 ? u : u3;
    };
    const int64_t umax = per_d(X, K, X);
    const int64_t ecap = X * X * X * X;
    if (pCap < umax || pLimit != purity_limit) {  // size the chunk buffers (first call or new limit)
      pLimit = purity_limit;
      size_t fr = 0, tot = 0;
      CK(cudaMemGetInfo(&fr, &tot));
      if (pX) cudaFree(pX);
      if (pP) cudaFree(pP);
      pX = pP = nullptr;
      double budget = 0.35 * (double)fr - 2.0 * (double)ecap * sizeof(C);  // per buffer
      if (purity_limit > 0) budget = (double)purity_limit / 2.0;
      int64_t dc = (int64_t)(budget / ((double)umax * sizeof(C)));
      if (dc < 1) return MPDO_ENOMEM;
      if (dc > X) dc = X;
      CK(dmalloc(&pX, dc * umax));
      CK(dmalloc(&pP, dc * umax));
      pCap = dc * umax;
    }
    if (pECap < ecap) {
      if (pE) cudaFree(pE);
      if (pE2) cudaFree(pE2);
      pE = pE2 = nullptr;
      CK(dmalloc(&pE, ecap));
      CK(dmalloc(&pE2, ecap));
      pECap = ecap;
    }
    out.assign(B, 0);
    for (int b = 0; b < B; ++b) {
      CK(fill<R>(stream, 1, pE, mk<R>(1, 0)));
      ++launches;
      for (int q = 0; q < n; ++q) {
        const int D = bond[q], dn = kraus[q], dr = bond[q + 1];
        const C* A = site_ptr(q) + (int64_t)b * slot_elems;
        const int64_t D2 = (int64_t)D * D, D3 = D2 * D;
        const int PN = 2 * dn * dr;
        int64_t Dc = pCap / per_d(D, dn, dr);
        if (Dc > D) Dc = D;
        for (int d0 = 0; d0 < D; d0 += (int)Dc) {
          const int dc = (int)(D - d0 < Dc ? D - d0 : Dc);
          // X1[(b,c,dd)][(p,n,r)] = sum_a E[a][b][c][d0 + dd] A[a][(p,n,r)]
          mpdo_status st = gemm_((int)(D2 * dc), PN, D, pE + d0, v2(0, dc, D, 1, 0, 0, D3), A, row_major(PN, 0), pX,
                                 row_major(PN, 0), 1);
          if (st) return st;
          // P1[c,dd,p,r,b,n] from X1[b,c,dd,p,n,r]
          {
            int dims[6] = {D, D, dc, 2, dn, dr};
            int perm[6] = {1, 2, 3, 5, 0, 4};
            CK(permute<R>(stream, 1, 6, dims, perm, pX, 0, pP, 0));
            ++launches;
          }
          // X2[(c,dd,p,r)][(q,s)] = sum_{(b,n)} P1[(c,dd,p,r)][(b,n)] conj(A[b,q,n,s])
          const int64_t M2 = (int64_t)D * dc * 2 * dr;
          st = gemm_((int)M2, 2 * dr, D * dn, pP, row_major((int64_t)D * dn, 0), A,
                     v2(0, dn, (int64_t)2 * dn * dr, dr, dr, (int64_t)dn * dr, 1, 1), pX, row_major(2 * dr, 0), 1);
          if (st) return st;
          // P2[dd,p,r,s,c,q] from X2[c,dd,p,r,q,s]
          {
            int dims[6] = {D, dc, 2, dr, 2, dr};
            int perm[6] = {1, 2, 3, 5, 0, 4};
            CK(permute<R>(stream, 1, 6, dims, perm, pX, 0, pP, 0));
            ++launches;
          }
          // X3[(dd,p,r,s)][(m,t)] = sum_{(c,q)} P2[(dd,p,r,s)][(c,q)] A[(c,q)][(m,t)]
          const int64_t M3 = (int64_t)dc * 2 * dr * dr;
          st = gemm_((int)M3, dn * dr, 2 * D, pP, row_major(2 * D, 0), A, row_major((int64_t)dn * dr, 0), pX,
                     row_major((int64_t)dn * dr, 0), 1);
          if (st) return st;
          // P3[r,s,t,dd,p,m] from X3[dd,p,r,s,m,t]
          {
            int dims[6] = {dc, 2, dr, dr, dn, dr};
            int perm[6] = {2, 3, 5, 0, 1, 4};
            CK(permute<R>(stream, 1, 6, dims, perm, pX, 0, pP, 0));
            ++launches;
          }
          // E'[(r,s,t)][u] (+)= sum_{(dd,p,m)} P3[(r,s,t)][(dd,p,m)] conj(A[(d0 + dd, p, m)][u])
          const int64_t M4 = (int64_t)dr * dr * dr;
          st = gemm_((int)M4, dr, dc * 2 * dn, pP, row_major((int64_t)dc * 2 * dn, 0), A + (int64_t)d0 * 2 * dn * dr,
                     v2(0, 0, 0, dr, 0, 0, 1, 1), pE2, row_major(dr, 0), 1, 0, d0 > 0);
          if (st) return st;
        }
        std::swap(pE, pE2);
      }
      C h;
      CK(cudaMemcpyAsync(&h, pE, sizeof(C), cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      out[b] = (double)h.x;
    }
    return MPDO_OK;
  }

  mpdo_status expect(int kind, const int* args, int nargs, double* out) override {
    if (capturing) return MPDO_ESTATE;
    {
      mpdo_status ss = read_status();
      if (ss) return ss;
    }
    if (kind == MPDO_EXPECT_DISCARDED) {
      CK(cudaMemcpyAsync(out, dDisc, sizeof(double) * 3 * B, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      return MPDO_OK;
    }
    if (kind == MPDO_EXPECT_DIMS) {
      for (int q = 1; q < n; ++q) out[q - 1] = bond[q];
      for (int q = 0; q < n; ++q) out[n - 1 + q] = kraus[q];
      return MPDO_OK;
    }
    mpdo_status st = build_envs();
    if (st) return st;
    std::vector<double> tr;
    if ((st = trace_(tr))) return st;
    auto finite = [&](double v) { return std::isfinite(v); };
    if (kind == MPDO_EXPECT_TRACE) {
      std::vector<int> ex(B);
      CK(cudaMemcpyAsync(ex.data(), dExp2, sizeof(int) * B, cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      for (int b = 0; b < B; ++b) out[b] = std::ldexp(tr[b], ex[b]);
      return MPDO_OK;
    }
    if (kind == MPDO_EXPECT_ZZ || kind == MPDO_EXPECT_ZZ_MAP || kind == MPDO_EXPECT_MAXCUT) {
      std::vector<std::pair<int, int>> pairs;
      if (kind == MPDO_EXPECT_ZZ) {
        if (nargs != 2 || !args) return MPDO_EINVAL;
        int i = args[0], j = args[1];
        if (i < 0 || j < 0 || i >= n || j >= n) return MPDO_EINVAL;
        if (i == j) {
          for (int b = 0; b < B; ++b) out[b] = 1.0;
          return MPDO_OK;
        }
        pairs.push_back({i < j ? i : j, i < j ? j : i});
      } else if (kind == MPDO_EXPECT_ZZ_MAP) {
        for (int i = 0; i < n; ++i)
          for (int j = i + 1; j < n; ++j) pairs.push_back({i, j});
      } else {
        if (nargs % 2 || (nargs && !args)) return MPDO_EINVAL;
        for (int e = 0; e < nargs / 2; ++e) {
          int i = args[2 * e], j = args[2 * e + 1];
          if (i < 0 || j < 0 || i >= n || j >= n || i == j) return MPDO_EINVAL;
          pairs.push_back({i < j ? i : j, i < j ? j : i});
        }
      }
      std::vector<std::vector<double>> vals;
      if ((st = zz_pairs(pairs, vals))) return st;
      if (kind == MPDO_EXPECT_ZZ) {
        for (int b = 0; b < B; ++b) out[b] = vals[0][b] / tr[b];
      } else if (kind == MPDO_EXPECT_ZZ_MAP) {
        for (int b = 0; b < B; ++b)
          for (int i = 0; i < n; ++i) out[(int64_t)b * n * n + i * n + i] = 1.0;
        for (size_t t = 0; t < pairs.size(); ++t)
          for (int b = 0; b < B; ++b) {
            double v = vals[t][b] / tr[b];
            out[(int64_t)b * n * n + pairs[t].first * n + pairs[t].second] = v;
            out[(int64_t)b * n * n + pairs[t].second * n + pairs[t].first] = v;
          }
      } else {
        for (int b = 0; b < B; ++b) {
          double s = 0;
          for (size_t t = 0; t < pairs.size(); ++t) s += 0.5 * (1.0 - vals[t][b] / tr[b]);
          out[b] = s;
        }
      }
      for (int b = 0; b < B; ++b)
        if (!finite(out[b])) return MPDO_ENOCONV;
      return MPDO_OK;
    }
    if (kind == MPDO_EXPECT_GHZ) {
      std::vector<double> r00, i00, r11, i11, r01, i01;
      if ((st = element_(0, 0, r00, i00)) || (st = element_(1, 1, r11, i11)) || (st = element_(0, 1, r01, i01)))
        return st;
      for (int b = 0; b < B; ++b) {
        out[b] = 0.5 * (r00[b] + r11[b] + 2 * r01[b]) / tr[b];
        if (!finite(out[b])) return MPDO_ENOCONV;
      }
      return MPDO_OK;
    }
    if (kind == MPDO_EXPECT_PROB) {
      if (nargs != n || !args) return MPDO_EINVAL;
      std::vector<int> z(args, args + n);
      for (int v : z)
        if (v != 0 && v != 1) return MPDO_EINVAL;
      std::vector<double> re, im;
      if ((st = element_bits(z, z, re, im))) return st;
      for (int b = 0; b < B; ++b) {
        out[b] = re[b] / tr[b];
        if (!finite(out[b])) return MPDO_ENOCONV;
      }
      return MPDO_OK;
    }
    if (kind == MPDO_EXPECT_PURITY) {
      std::vector<double> p;
      if ((st = purity_(p))) return st;
      for (int b = 0; b < B; ++b) {
        out[b] = p[b] / (tr[b] * tr[b]);
        if (!finite(out[b])) return MPDO_ENOCONV;
      }
      return MPDO_OK;
    }
    return MPDO_EINVAL;
  }

  // put every site back into the slot and centre it had at capture begin (dims must match)
  mpdo_status restore_layout() override {
    for (int q = 0; q < n; ++q)
      if (bond[q] != snap_bond[q] || kraus[q] != snap_kraus[q]) return MPDO_ESTATE;
    mpdo_status st = move_centre(snap_centre);
    if (st) return st;
    // permutation of slots: copy site q from its current slot to snap_slot[q] through free slots
    std::vector<int> cur = site_slot;
    std::vector<int> owner(nslots, -1);
    for (int q = 0; q < n; ++q) owner[cur[q]] = q;
    for (int q = 0; q < n; ++q) {
      int target = snap_slot[q];
      if (cur[q] == target) continue;
      // if target is occupied by site p, move p to a free slot first
      int p = owner[target];
      if (p >= 0) {
        int f = -1;
        for (int s = 0; s < nslots; ++s)
          if (owner[s] < 0) {
            f = s;
            break;
          }
        CK(cudaMemcpyAsync(slot_ptr(f), slot_ptr(target), sizeof(C) * (size_t)B * slot_elems, cudaMemcpyDeviceToDevice,
                           stream));
        owner[f] = p;
        owner[target] = -1;
        cur[p] = f;
      }
      CK(cudaMemcpyAsync(slot_ptr(target), slot_ptr(cur[q]), sizeof(C) * (size_t)B * slot_elems,
                         cudaMemcpyDeviceToDevice, stream));
      owner[cur[q]] = -1;
      owner[target] = q;
      cur[q] = target;
    }
    site_slot = cur;
    free_slots.clear();
    for (int s = nslots - 1; s >= 0; --s)
      if (owner[s] < 0) free_slots.push_back(s);
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- site access
  mpdo_status get_site(int chain, int q, double* out) override {
    const int64_t cnt = (int64_t)bond[q] * 2 * kraus[q] * bond[q + 1];
    std::vector<C> h((size_t)cnt);
    CK(cudaMemcpyAsync(h.data(), site_ptr(q) + (int64_t)chain * slot_elems, sizeof(C) * cnt, cudaMemcpyDeviceToHost,
                       stream));
    CK(cudaStreamSynchronize(stream));
    for (int64_t i = 0; i < cnt; ++i) {
      out[2 * i] = (double)h[i].x;
      out[2 * i + 1] = (double)h[i].y;
    }
    return MPDO_OK;
  }
  mpdo_status set_site(int q, int dl, int dn, int dr, const double* data) override {
    const int64_t cnt = (int64_t)dl * 2 * dn * dr;
    std::vector<C> h((size_t)cnt * B);
    for (int b = 0; b < B; ++b)
      for (int64_t i = 0; i < cnt; ++i) h[b * cnt + i] = mk<R>((R)data[2 * (b * cnt + i)], (R)data[2 * (b * cnt + i) + 1]);
    CK(cudaStreamSynchronize(stream));
    for (int b = 0; b < B; ++b)
      CK(cudaMemcpy(site_ptr(q) + (int64_t)b * slot_elems, h.data() + b * cnt, sizeof(C) * cnt, cudaMemcpyHostToDevice));
    bond[q] = dl;
    bond[q + 1] = dr;
    kraus[q] = dn;
    return MPDO_OK;
  }

  // ---------------------------------------------------------------- checkpoint
  mpdo_status save(FILE* f) override {
    std::vector<C> h((size_t)B * slot_elems);
    for (int q = 0; q < n; ++q) {
      CK(cudaMemcpyAsync(h.data(), site_ptr(q), sizeof(C) * h.size(), cudaMemcpyDeviceToHost, stream));
      CK(cudaStreamSynchronize(stream));
      if (fwrite(h.data(), sizeof(C), h.size(), f) != h.size()) return MPDO_EINVAL;
    }
    std::vector<double> d(3 * (size_t)B);
    CK(cudaMemcpyAsync(d.data(), dDisc, sizeof(double) * d.size(), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (fwrite(d.data(), sizeof(double), d.size(), f) != d.size()) return MPDO_EINVAL;
    std::vector<int> ex(B);
    CK(cudaMemcpyAsync(ex.data(), dExp2, sizeof(int) * B, cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    if (fwrite(ex.data(), sizeof(int), ex.size(), f) != ex.size()) return MPDO_EINVAL;
    return MPDO_OK;
  }
  mpdo_status load(FILE* f) override {
    std::vector<C> h((size_t)B * slot_elems);
    for (int q = 0; q < n; ++q) {
      if (fread(h.data(), sizeof(C), h.size(), f) != h.size()) return MPDO_EINVAL;
      CK(cudaMemcpy(site_ptr(q), h.data(), sizeof(C) * h.size(), cudaMemcpyHostToDevice));
    }
    std::vector<double> d(3 * (size_t)B);
    if (fread(d.data(), sizeof(double), d.size(), f) != d.size()) return MPDO_EINVAL;
    CK(cudaMemcpy(dDisc, d.data(), sizeof(double) * d.size(), cudaMemcpyHostToDevice));
    std::vector<int> ex(B);
    if (fread(ex.data(), sizeof(int), ex.size(), f) != ex.size()) return MPDO_EINVAL;
    CK(cudaMemcpy(dExp2, ex.data(), sizeof(int) * ex.size(), cudaMemcpyHostToDevice));
    return MPDO_OK;
  }
};

EngBase* make_engine(int prec) {
  switch (prec) {
    case MPDO_FP64: return new (std::nothrow) Eng<double, double>();
    case MPDO_MIXED: return new (std::nothrow) Eng<float, double>();
    case MPDO_FP32: return new (std::nothrow) Eng<float, float>();
  }
  return nullptr;
}

}  // namespace

struct mpdo_ctx {
  EngBase* e = nullptr;
  double guard_tol = 0;             // trace guard: off when <= 0
  std::vector<double> guard_last;   // Tr rho of every chain after the previous guarded call
  ~mpdo_ctx() { delete e; }
};

// The trace guard after a gate or truncation that returned `st`: reads Tr rho of every chain and
// compares it with the reading after the previous guarded call.  The channels are trace preserving and
// truncations only drop weight, so a growth beyond the tolerance (or a negative or non-finite trace)
// means the call went wrong.  A trace that underflowed to 0 passes.
static mpdo_status guard_after(mpdo_ctx* h, mpdo_status st) {
  if (st != MPDO_OK || !(h->guard_tol > 0) || h->e->capturing) return st;
  std::vector<double> tr(h->e->B);
  st = h->e->expect(MPDO_EXPECT_TRACE, nullptr, 0, tr.data());
  if (st) return st;
  bool bad = false;
  for (int b = 0; b < h->e->B; ++b)
    if (!(tr[b] >= 0) || !std::isfinite(tr[b]) || tr[b] > h->guard_last[b] * (1.0 + h->guard_tol)) bad = true;
  h->guard_last = tr;
  return bad ? MPDO_EDRIFT : MPDO_OK;
}

// ====================================================================== C ABI
extern "C" {

const char* mpdo_status_string(int s) {
  switch (s) {
    case MPDO_OK: return "ok";
    case MPDO_EINVAL: return "invalid argument";
    case MPDO_ENOMEM: return "out of memory";
    case MPDO_ENOTCP: return "process matrix is not completely positive";
    case MPDO_ENOTTP: return "process matrix is not trace preserving";
    case MPDO_ENOCONV: return "eigensolver or readout produced a non-finite or collapsed result";
    case MPDO_ETIMEOUT: return "timeout";
    case MPDO_ECUDA: return "CUDA error";
    case MPDO_ESTATE: return "invalid state for this call";
    case MPDO_EDRIFT: return "trace guard: Tr rho grew or became non-finite";
  }
  return "unknown status";
}

mpdo_status mpdo_init_batch(int batch, int n, int chi_max, int kappa_max, int prec, void* stream, mpdo_t* out) {
  if (!out || batch < 1 || n < 1 || chi_max < 1 || kappa_max < 1 || batch > 65535) return MPDO_EINVAL;
  if (4 * chi_max > 512 || 16 * kappa_max > 512) return MPDO_EINVAL;  // eigensolver size limit
  if (prec != MPDO_FP64 && prec != MPDO_MIXED && prec != MPDO_FP32) return MPDO_EINVAL;
  mpdo_ctx* h = new (std::nothrow) mpdo_ctx();
  if (!h) return MPDO_ENOMEM;
  h->e = make_engine(prec);
  if (!h->e) {
    delete h;
    return MPDO_ENOMEM;
  }
  EngBase* e = h->e;
  e->B = batch;
  e->n = n;
  e->chi_max = chi_max;
  e->kappa_max = kappa_max;
  e->prec = prec;
  e->stream = (cudaStream_t)stream;
  cudaGetDevice(&e->device);
  mpdo_status st = e->alloc();
  if (st) {
    cudaError_t le = e->last_err;
    delete h;
    return le == cudaErrorMemoryAllocation ? MPDO_ENOMEM : st;
  }
  *out = h;
  return MPDO_OK;
}

mpdo_status mpdo_init(int n, int chi_max, int kappa_max, int prec, void* stream, mpdo_t* out) {
  return mpdo_init_batch(1, n, chi_max, kappa_max, prec, stream, out);
}

mpdo_status mpdo_free(mpdo_t h) {
  if (!h) return MPDO_EINVAL;
  if (h->e && h->e->capturing) return MPDO_ESTATE;
  if (h->e) cudaStreamSynchronize(h->e->stream);
  delete h;
  return MPDO_OK;
}

mpdo_status mpdo_reset(mpdo_t h) {
  if (!h) return MPDO_EINVAL;
  mpdo_status st = h->e->reset();
  if (st == MPDO_OK && h->guard_tol > 0) h->guard_last.assign(h->e->B, 1.0);
  return st;
}

mpdo_status mpdo_sync(mpdo_t h) {
  if (!h) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  return h->e->sync();
}

mpdo_status channel_set_from_process_matrices(mpdo_t h, int nq, int count, const double* chi, double tol,
                                              mpdo_chan_t* out, int* n_kraus) {
  if (!h || !out || !chi || count < 1 || nq < 1 || nq > 3) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  if (!(tol > 0)) tol = 1e-12;
  const int d = 1 << nq, d2 = d * d;
  const int64_t per = (int64_t)d2 * d2;
  // host checks: finite, Hermitian, trace 1
  for (int c = 0; c < count; ++c) {
    const double* X = chi + 2 * per * c;
    double tr_re = 0, tr_im = 0;
    for (int a = 0; a < d2; ++a)
      for (int b = 0; b < d2; ++b) {
        double re = X[2 * (a * d2 + b)], im = X[2 * (a * d2 + b) + 1];
        double re2 = X[2 * (b * d2 + a)], im2 = X[2 * (b * d2 + a) + 1];
        if (!std::isfinite(re) || !std::isfinite(im)) return MPDO_EINVAL;
        if (std::fabs(re - re2) > 1e-10 || std::fabs(im + im2) > 1e-10) return MPDO_EINVAL;
        if (a == b) {
          tr_re += re;
          tr_im += im;
        }
      }
    if (std::fabs(tr_re - 1.0) > 1e-8 || std::fabs(tr_im) > 1e-8) return MPDO_ENOTTP;
  }
  cudaStream_t s = h->e->stream;
  cplx<double>*dchi = nullptr, *dchoi = nullptr, *dvec = nullptr;
  double *deta = nullptr, *dscr = nullptr, *derr = nullptr;
  int* dr = nullptr;
  const int64_t scr = eig_scratch_elems(d2, d2);
  mpdo_status ret = MPDO_OK;
  std::unique_ptr<mpdo_chanset> cs(new (std::nothrow) mpdo_chanset());
  if (!cs) return MPDO_ENOMEM;
  std::vector<double> eta((size_t)count * d2);
  std::vector<int> ranks(count);
  int rmax = 1;
  auto fail = [&](mpdo_status st) {
    ret = st;
    return st;
  };
  do {
    if (cudaMalloc((void**)&dchi, sizeof(cplx<double>) * per * count) != cudaSuccess ||
        cudaMalloc((void**)&dchoi, sizeof(cplx<double>) * per * count) != cudaSuccess ||
        cudaMalloc((void**)&dvec, sizeof(cplx<double>) * per * count) != cudaSuccess ||
        cudaMalloc((void**)&deta, sizeof(double) * d2 * count) != cudaSuccess ||
        cudaMalloc((void**)&dscr, sizeof(double) * scr * count) != cudaSuccess ||
        cudaMalloc((void**)&derr, sizeof(double) * count) != cudaSuccess ||
        cudaMalloc((void**)&dr, sizeof(int) * count) != cudaSuccess) {
      fail(MPDO_ENOMEM);
      break;
    }
    if (cudaMemcpyAsync(dchi, chi, sizeof(cplx<double>) * per * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        chi_to_choi(s, count, nq, dchi, dchoi) != cudaSuccess) {
      fail(MPDO_ECUDA);
      break;
    }
    EigArgs<double> a;
    a.A = dchoi;
    a.astride = per;
    a.n = d2;
    a.k = d2;
    a.w = deta;
    a.wstride = d2;
    a.V = dvec;
    a.vv = col_major(d2, per);
    a.scratch = dscr;
    a.sstride = scr;
    a.disc = nullptr;
    a.gap = nullptr;
    a.disc_stride = 0;
    if (heevk<double>(s, count, a) != cudaSuccess ||
        cudaMemcpyAsync(eta.data(), deta, sizeof(double) * d2 * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      fail(MPDO_ECUDA);
      break;
    }
    h->e->launches += 2;
    for (int c = 0; c < count && !ret; ++c) {
      const double* w = &eta[(size_t)c * d2];
      double neg = 0, emax = w[0] > 0 ? w[0] : 0;
      for (int i = 0; i < d2; ++i)
        if (w[i] < 0) neg -= w[i];
      if (neg > 1e-8) {
        fail(MPDO_ENOTCP);
        break;
      }
      int r = 0;
      for (int i = 0; i < d2; ++i)
        if (w[i] > tol * emax && w[i] > 0) ++r;
      if (r < 1) r = 1;
      ranks[c] = r;
      rmax = r > rmax ? r : rmax;
    }
    if (ret) break;
    if (cudaMalloc((void**)&cs->kraus, sizeof(cplx<double>) * (size_t)count * rmax * d * d) != cudaSuccess) {
      fail(MPDO_ENOMEM);
      break;
    }
    std::vector<double> err(count);
    if (cudaMemcpyAsync(dr, ranks.data(), sizeof(int) * count, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        choi_to_kraus(s, count, nq, rmax, dr, deta, dvec, cs->kraus) != cudaSuccess ||
        kraus_tp_error(s, count, nq, rmax, cs->kraus, derr) != cudaSuccess ||
        cudaMemcpyAsync(err.data(), derr, sizeof(double) * count, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      fail(MPDO_ECUDA);
      break;
    }
    h->e->launches += 2;
    for (int c = 0; c < count; ++c)
      if (!(err[c] <= 1e-8)) {
        fail(MPDO_ENOTTP);
        break;
      }
  } while (0);
  cudaFree(dchi);
  cudaFree(dchoi);
  cudaFree(dvec);
  cudaFree(deta);
  cudaFree(dscr);
  cudaFree(derr);
  cudaFree(dr);
  if (ret) return ret;
  cs->nq = nq;
  cs->count = count;
  cs->rpad = rmax;
  cs->device = h->e->device;
  cs->ranks = ranks;
  if (n_kraus)
    for (int c = 0; c < count; ++c) n_kraus[c] = ranks[c];
  *out = cs.release();
  return MPDO_OK;
}

mpdo_status channel_from_process_matrix(mpdo_t h, int nq, const double* chi, double tol, mpdo_chan_t* out,
                                        int* n_kraus) {
  return channel_set_from_process_matrices(h, nq, 1, chi, tol, out, n_kraus);
}

mpdo_status channel_kraus(mpdo_chan_t ch, int idx, double* out, int* r_pad) {
  if (!ch || idx < 0 || idx >= ch->count || !out) return MPDO_EINVAL;
  const int d = 1 << ch->nq;
  const size_t cnt = (size_t)ch->rpad * d * d;
  if (cudaMemcpy(out, ch->kraus + (int64_t)idx * cnt, sizeof(cplx<double>) * cnt, cudaMemcpyDeviceToHost) !=
      cudaSuccess)
    return MPDO_ECUDA;
  if (r_pad) *r_pad = ch->rpad;
  return MPDO_OK;
}

mpdo_status channel_free(mpdo_chan_t ch) {
  if (!ch) return MPDO_EINVAL;
  cudaDeviceSynchronize();
  delete ch;
  return MPDO_OK;
}

mpdo_status apply_1q(mpdo_t h, int q, const double* U, mpdo_chan_t ch) {
  if (!h || !U) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(1, q, U, nullptr, ch, nullptr));
}
mpdo_status apply_2q(mpdo_t h, int q, const double* U, mpdo_chan_t ch) {
  if (!h || !U) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(2, q, U, nullptr, ch, nullptr));
}
mpdo_status apply_3q(mpdo_t h, int q, const double* U, mpdo_chan_t ch) {
  if (!h || !U) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(3, q, U, nullptr, ch, nullptr));
}
mpdo_status apply_3q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev) {
  if (!h || !U_dev) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(3, q, nullptr, U_dev, ch, chan_idx_dev));
}
mpdo_status apply_1q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev) {
  if (!h || !U_dev) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(1, q, nullptr, U_dev, ch, chan_idx_dev));
}
mpdo_status apply_2q_batch(mpdo_t h, int q, const double* U_dev, mpdo_chan_t ch, const int* chan_idx_dev) {
  if (!h || !U_dev) return MPDO_EINVAL;
  return guard_after(h, h->e->apply(2, q, nullptr, U_dev, ch, chan_idx_dev));
}
mpdo_status truncate_kraus(mpdo_t h, int q, int kappa, double* discarded) {
  if (!h) return MPDO_EINVAL;
  if (discarded && h->e->capturing) return MPDO_ESTATE;
  return guard_after(h, h->e->truncate(q, kappa, discarded));
}
mpdo_status truncate_bonds(mpdo_t h, int chi, double* discarded) {
  if (!h) return MPDO_EINVAL;
  if (discarded && h->e->capturing) return MPDO_ESTATE;
  return guard_after(h, h->e->truncate_bonds(chi, discarded));
}
mpdo_status mpdo_distribution(mpdo_t h, double* out) {
  if (!h || !out) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  return h->e->distribution(out);
}
mpdo_status mpdo_jsd(const double* p, const double* q, int len, double* out) {
  if (!p || !q || !out || len < 1) return MPDO_EINVAL;
  double sp = 0, sq = 0;
  for (int i = 0; i < len; ++i) {
    if (!(p[i] >= 0) || !(q[i] >= 0) || !std::isfinite(p[i]) || !std::isfinite(q[i])) return MPDO_EINVAL;
    sp += p[i];
    sq += q[i];
  }
  if (!(sp > 0) || !(sq > 0)) return MPDO_EINVAL;
  // JSD = (KL(p || m) + KL(q || m)) / 2 with m = (p + q) / 2, natural log, 0 log 0 = 0
  double js = 0;
  for (int i = 0; i < len; ++i) {
    const double a = p[i] / sp, b = q[i] / sq, m = 0.5 * (a + b);
    if (a > 0) js += 0.5 * a * std::log(a / m);
    if (b > 0) js += 0.5 * b * std::log(b / m);
  }
  *out = js;
  return MPDO_OK;
}
mpdo_status expect(mpdo_t h, int kind, const int* args, int nargs, double* out) {
  if (!h || !out) return MPDO_EINVAL;
  return h->e->expect(kind, args, nargs, out);
}

static const char kMagic[8] = {'M', 'P', 'D', 'O', 'C', 'K', 'P', '2'};

mpdo_status mpdo_save(mpdo_t h, const char* path) {
  if (!h || !path) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  // canonical layout: centre first to 0 is not needed; store dims and centre as they are
  mpdo_status cst = e->clean();
  if (cst) return cst;
  FILE* f = fopen(path, "wb");
  if (!f) return MPDO_EINVAL;
  int hdr[6] = {e->B, e->n, e->chi_max, e->kappa_max, e->prec, e->centre};
  bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 6, f) == 6 &&
            fwrite(e->bond.data(), sizeof(int), e->n + 1, f) == (size_t)e->n + 1 &&
            fwrite(e->kraus.data(), sizeof(int), e->n, f) == (size_t)e->n;
  mpdo_status st = ok ? e->save(f) : MPDO_EINVAL;
  fclose(f);
  return st;
}

mpdo_status mpdo_load(const char* path, void* stream, mpdo_t* out) {
  if (!path || !out) return MPDO_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return MPDO_EINVAL;
  char magic[8];
  int hdr[6];
  if (fread(magic, 1, 8, f) != 8 || std::memcmp(magic, kMagic, 8) != 0 || fread(hdr, sizeof(int), 6, f) != 6) {
    fclose(f);
    return MPDO_EINVAL;
  }
  mpdo_t h = nullptr;
  mpdo_status st = mpdo_init_batch(hdr[0], hdr[1], hdr[2], hdr[3], hdr[4], stream, &h);
  if (st) {
    fclose(f);
    return st;
  }
  EngBase* e = h->e;
  e->centre = hdr[5];
  bool ok = fread(e->bond.data(), sizeof(int), e->n + 1, f) == (size_t)e->n + 1 &&
            fread(e->kraus.data(), sizeof(int), e->n, f) == (size_t)e->n;
  st = ok ? e->load(f) : MPDO_EINVAL;
  fclose(f);
  if (st) {
    mpdo_free(h);
    return st;
  }
  *out = h;
  return MPDO_OK;
}

mpdo_status mpdo_capture_begin(mpdo_t h) {
  if (!h) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  if (e->stream == nullptr) return MPDO_ESTATE;  // the legacy stream cannot be captured
  mpdo_status cst = e->clean();
  if (cst) return cst;
  if (cudaStreamSynchronize(e->stream) != cudaSuccess) return MPDO_ECUDA;
  e->snap_bond = e->bond;
  e->snap_kraus = e->kraus;
  e->snap_slot = e->slots();
  e->snap_centre = e->centre;
  if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return MPDO_ECUDA;
  e->capturing = true;
  return MPDO_OK;
}

mpdo_status mpdo_capture_end(mpdo_t h, int restore, mpdo_graph_t* out) {
  if (!h || !out) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (!e->capturing) return MPDO_ESTATE;
  mpdo_status st = MPDO_OK;
  if (restore) st = e->restore_layout();
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(e->stream, &g);
  e->capturing = false;
  if (st) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return MPDO_ECUDA;
  mpdo_graph* gr = new (std::nothrow) mpdo_graph();
  if (!gr) {
    cudaGraphDestroy(g);
    return MPDO_ENOMEM;
  }
  gr->graph = g;
  gr->stream = e->stream;
  if (cudaGraphInstantiate(&gr->exec, g, 0) != cudaSuccess) {
    delete gr;
    return MPDO_ECUDA;
  }
  *out = gr;
  return MPDO_OK;
}

mpdo_status mpdo_graph_launch(mpdo_graph_t g) {
  if (!g) return MPDO_EINVAL;
  return cudaGraphLaunch(g->exec, g->stream) == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
}

mpdo_status mpdo_graph_free(mpdo_graph_t g) {
  if (!g) return MPDO_EINVAL;
  cudaStreamSynchronize(g->stream);
  delete g;
  return MPDO_OK;
}

mpdo_status mpdo_get_site(mpdo_t h, int chain, int q, double* out, int* dims) {
  if (!h || !out) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  if (chain < 0 || chain >= e->B || q < 0 || q >= e->n) return MPDO_EINVAL;
  if (dims) {
    dims[0] = e->bond[q];
    dims[1] = e->kraus[q];
    dims[2] = e->bond[q + 1];
  }
  return e->get_site(chain, q, out);
}

mpdo_status mpdo_set_site(mpdo_t h, int q, int dl, int dn, int dr, const double* data) {
  if (!h || !data) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  if (q < 0 || q >= e->n || dl < 1 || dn < 1 || dr < 1 || dl > e->chi_max || dr > e->chi_max || dn > e->kappa_max)
    return MPDO_EINVAL;
  if ((q == 0 && dl != 1) || (q == e->n - 1 && dr != 1)) return MPDO_EINVAL;
  return e->set_site(q, dl, dn, dr, data);
}

mpdo_status mpdo_set_centre(mpdo_t h, int q) {
  if (!h) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  if (q < 0 || q >= h->e->n) return MPDO_EINVAL;
  h->e->centre = q;
  h->e->dirty = -1;
  return MPDO_OK;
}

mpdo_status mpdo_set_tensor_cores(mpdo_t h, int enable) {
  if (!h) return MPDO_EINVAL;
  if (enable && h->e->prec != MPDO_FP64) {
    if (h->e->capturing) return MPDO_ESTATE;
    mpdo_status st = h->e->alloc_tc();
    if (st) return st;
  }
  h->e->tensor_cores = enable != 0;
  return MPDO_OK;
}

// Uhlmann fidelity F(rho, sigma) = (tr sqrt(sqrt(rho) sigma sqrt(rho)))^2 of chain ca of a and chain cb
// of b (Sec. IV.C), both normalised to unit trace, in FP64 on a's stream.  Each chain's dense density
// matrix comes from its sites by the contraction of Sec. II.C (stored row-major, i.e. its complex
// conjugate read column-major, which leaves F unchanged); sqrt(rho) = Y Y^H with Y = V diag(lambda^1/4)
// from rho's eigendecomposition; F = (sum sqrt(mu))^2 / (tr rho tr sigma) over the eigenvalues mu of
// sqrt(rho) sigma sqrt(rho).
mpdo_status mpdo_fidelity(mpdo_t a, int ca, mpdo_t b, int cb, double* out) {
  if (!a || !b || !out) return MPDO_EINVAL;
  EngBase *ea = a->e, *eb = b->e;
  if (ea->capturing || eb->capturing) return MPDO_ESTATE;
  if (ea->n != eb->n || ea->n > 7 || ca < 0 || ca >= ea->B || cb < 0 || cb >= eb->B) return MPDO_EINVAL;
  mpdo_status st = ea->clean();
  if (!st) st = eb->clean();
  if (!st) st = ea->sync();
  if (!st) st = eb->sync();
  if (st) return st;
  const int N = 1 << ea->n;
  const int64_t work = lmax(lmax(ea->dense_work(), eb->dense_work()), (int64_t)N * N);
  if (work > ((int64_t)1 << 27)) return MPDO_EINVAL;  // intermediates of at most 2 GB each
  const int64_t site = lmax(2LL * ea->kappa_max * ea->chi_max * ea->chi_max, 2LL * eb->kappa_max * eb->chi_max * eb->chi_max);
  cudaStream_t s = ea->stream;
  cplx<double>*X = nullptr, *Y = nullptr, *S = nullptr, *rho = nullptr, *sig = nullptr, *V = nullptr, *T1 = nullptr,
               *T2 = nullptr;
  double *w = nullptr, *scr = nullptr;
  const int64_t NN = (int64_t)N * N, sc = eig_scratch_elems(N, N);
  auto ok = [](cudaError_t e) { return e == cudaSuccess; };
  bool good = ok(cudaMalloc((void**)&X, sizeof(cplx<double>) * work)) &&
              ok(cudaMalloc((void**)&Y, sizeof(cplx<double>) * work)) && ok(cudaMalloc((void**)&S, sizeof(cplx<double>) * site)) &&
              ok(cudaMalloc((void**)&rho, sizeof(cplx<double>) * NN)) && ok(cudaMalloc((void**)&sig, sizeof(cplx<double>) * NN)) &&
              ok(cudaMalloc((void**)&V, sizeof(cplx<double>) * NN)) && ok(cudaMalloc((void**)&T1, sizeof(cplx<double>) * NN)) &&
              ok(cudaMalloc((void**)&T2, sizeof(cplx<double>) * NN)) && ok(cudaMalloc((void**)&w, sizeof(double) * N)) &&
              ok(cudaMalloc((void**)&scr, sizeof(double) * sc));
  st = good ? MPDO_OK : MPDO_ENOMEM;
  auto gemm64 = [&](int M, int Nn, int K, const cplx<double>* A, View va, const cplx<double>* Bm, View vb, cplx<double>* C,
                    View vc) {
    GemmArgs<double> g;
    g.M = M;
    g.N = Nn;
    g.K = K;
    g.alpha = mk<double>(1, 0);
    g.beta = mk<double>(0, 0);
    g.A = A;
    g.va = va;
    g.B = Bm;
    g.vb = vb;
    g.C = C;
    g.vc = vc;
    return gemm<double>(s, 1, g) == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
  };
  auto eig = [&](cplx<double>* A) {
    EigArgs<double> e;
    e.A = A;
    e.astride = NN;
    e.n = N;
    e.k = N;
    e.w = w;
    e.wstride = N;
    e.V = V;
    e.vv = col_major(N, NN);
    e.scratch = scr;
    e.sstride = sc;
    e.disc = nullptr;
    e.gap = nullptr;
    e.disc_stride = 0;
    return heevk<double>(s, 1, e) == cudaSuccess ? MPDO_OK : MPDO_ECUDA;
  };
  std::vector<double> hw(N), hs(N), hmu(N);
  std::vector<cplx<double>> hsig((size_t)NN);
  if (!st) st = ea->dense_rho(ca, s, X, Y, S);
  if (!st && cudaMemcpyAsync(rho, X, sizeof(cplx<double>) * NN, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = MPDO_ECUDA;
  if (!st) st = eb->dense_rho(cb, s, X, Y, S);
  if (!st && cudaMemcpyAsync(sig, X, sizeof(cplx<double>) * NN, cudaMemcpyDeviceToDevice, s) != cudaSuccess) st = MPDO_ECUDA;
  if (!st && cudaMemcpyAsync(hsig.data(), sig, sizeof(cplx<double>) * NN, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    st = MPDO_ECUDA;
  // Y = V diag(lambda^1/4), sqrt(rho) = Y Y^H
  if (!st) st = eig(rho);
  if (!st && (cudaMemcpyAsync(hw.data(), w, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    st = MPDO_ECUDA;
  double tr_rho = 0, tr_sig = 0;
  if (!st) {
    for (int i = 0; i < N; ++i) {
      tr_rho += hw[i];
      tr_sig += hsig[(size_t)i * N + i].x;
      hs[i] = std::sqrt(std::sqrt(hw[i] > 0 ? hw[i] : 0.0));
    }
    if (cudaMemcpyAsync(w, hs.data(), sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        scale_cols(s, N, V, w) != cudaSuccess)
      st = MPDO_ECUDA;
  }
  if (!st) st = gemm64(N, N, N, V, col_major(N, 0), V, v2(0, 0, 0, N, 0, 0, 1, 1), T1, col_major(N, 0));  // sqrt(rho)
  if (!st) st = gemm64(N, N, N, T1, col_major(N, 0), sig, col_major(N, 0), T2, col_major(N, 0));
  if (!st) st = gemm64(N, N, N, T2, col_major(N, 0), T1, col_major(N, 0), rho, col_major(N, 0));
  if (!st) st = eig(rho);
  if (!st && (cudaMemcpyAsync(hmu.data(), w, sizeof(double) * N, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
              cudaStreamSynchronize(s) != cudaSuccess))
    st = MPDO_ECUDA;
  for (void* p : {(void*)X, (void*)Y, (void*)S, (void*)rho, (void*)sig, (void*)V, (void*)T1, (void*)T2, (void*)w, (void*)scr})
    if (p) cudaFree(p);
  if (st) return st;
  double f = 0;
  for (int i = 0; i < N; ++i) f += std::sqrt(hmu[i] > 0 ? hmu[i] : 0.0);
  f = f * f / (tr_rho * tr_sig);
  if (!std::isfinite(f)) return MPDO_ENOCONV;
  *out = f;
  return MPDO_OK;
}

mpdo_status mpdo_set_trunc_order(mpdo_t h, int order) {
  if (!h || (order != MPDO_TRUNC_SPLIT_FIRST && order != MPDO_TRUNC_KRAUS_FIRST)) return MPDO_EINVAL;
  h->e->trunc_order = order;
  return MPDO_OK;
}

mpdo_status mpdo_set_neighbour_truncation(mpdo_t h, int enable) {
  if (!h) return MPDO_EINVAL;
  h->e->neighbour_trunc = enable != 0;
  return MPDO_OK;
}

mpdo_status mpdo_set_trace_guard(mpdo_t h, double tol) {
  if (!h || std::isnan(tol)) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  if (!(tol > 0)) {
    h->guard_tol = 0;
    h->guard_last.clear();
    return MPDO_OK;
  }
  std::vector<double> tr(h->e->B);
  mpdo_status st = h->e->expect(MPDO_EXPECT_TRACE, nullptr, 0, tr.data());
  if (st) return st;
  h->guard_tol = tol;
  h->guard_last = tr;
  return MPDO_OK;
}

mpdo_status mpdo_set_purity_memory(mpdo_t h, long long bytes) {
  if (!h || bytes < 0) return MPDO_EINVAL;
  if (h->e->capturing) return MPDO_ESTATE;
  h->e->purity_limit = bytes;
  return MPDO_OK;
}

mpdo_status mpdo_profile(mpdo_t h, int enable) {
  if (!h) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  if (enable && e->ev_pool.empty()) {
    e->ev_pool.resize(1 << 16);
    for (auto& ev : e->ev_pool)
      if (cudaEventCreate(&ev) != cudaSuccess) return MPDO_ECUDA;
  }
  e->prof_on = enable != 0;
  return MPDO_OK;
}

mpdo_status mpdo_profile_read(mpdo_t h, double* ms, double* flops, long long* count) {
  if (!h || !ms || !flops || !count) return MPDO_EINVAL;
  EngBase* e = h->e;
  if (e->capturing) return MPDO_ESTATE;
  if (cudaStreamSynchronize(e->stream) != cudaSuccess) return MPDO_ECUDA;
  for (int c = 0; c < EngBase::P_N; ++c) {
    ms[c] = 0;
    flops[c] = 0;
    count[c] = 0;
  }
  for (auto& r : e->recs) {
    float t = 0;
    if (cudaEventElapsedTime(&t, e->ev_pool[r.e0], e->ev_pool[r.e1]) != cudaSuccess) return MPDO_ECUDA;
    ms[r.cls] += t;
    flops[r.cls] += r.flops;
    count[r.cls] += 1;
    if (r.sub >= 0) {
      ms[r.sub] += t;
      flops[r.sub] += r.sub == EngBase::P_ONEQ ? r.bytes : r.flops;
      count[r.sub] += 1;
    }
  }
  e->recs.clear();
  e->ev_next = 0;
  return MPDO_OK;
}

long long mpdo_launch_count(mpdo_t h) { return h ? h->e->launches : -1; }

}  // extern "C"
