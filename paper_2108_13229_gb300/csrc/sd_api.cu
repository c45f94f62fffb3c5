// sd_api.cu -- host side of the C ABI (include/sd.h): device memory arena,
// multigrid hierarchy setup, the block preconditioner of Sec. 4 with
// geometric V-cycles for the V and D' blocks, the FP64 flexible GMRES(m)
// outer solve, the implicit-Euler time loop (Sec. 2), batched execution of
// independent instances and the continuous-batching server.
#include "../../include/sd.h"
#include "sd_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <type_traits>
#include <vector>

using namespace sdk;

namespace {

thread_local char g_errmsg[256];

#define CK(call)                                                                                 \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      snprintf(g_errmsg, sizeof(g_errmsg), "%s at %s:%d", cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? SD_E_NOMEM : SD_E_CUDA;                            \
    }                                                                                            \
  } while (0)

#define CKR(expr)              \
  do {                         \
    int r_ = (expr);           \
    if (r_ != SD_OK) return r_; \
  } while (0)

bool is_device_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------- arena
// Every buffer of a handle comes from one cudaMalloc; a planning pass sizes
// it, so sd_memory_estimate() reports exactly what sd_create() allocates.
struct Arena {
  char* base = nullptr;
  size_t off = 0;
  bool plan = true;
  template <typename T>
  T* take(long long count) {
    size_t bytes = ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
    T* p = plan ? nullptr : reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Work vectors of one block (V, D' or the pressure Laplacian P) on one level.
template <typename T>
struct Block {
  T *b = nullptr, *x = nullptr, *x2 = nullptr, *d = nullptr, *r = nullptr;
  T* res = nullptr;          // where the last V-cycle left its result
  std::vector<T> cha, chc;   // Chebyshev step coefficients
  T* cht = nullptr;          // the same in device memory: a at cht[0..7], c at cht[8..15]
};

// Coefficient arrays of one level (the Darcy set from K, the pressure
// Laplacian set from a unit permeability).  TyR (FP64 sets only): Ty of the
// preconditioner's Darcy block, whose top faces may carry the interface's
// Schur correction (sd_options.darcy_schur); the operator reads Ty.
template <typename T>
struct LevelCoef {
  T *w = nullptr, *rg = nullptr, *Tx = nullptr, *Ty = nullptr;
  T *wP = nullptr, *rgP = nullptr, *TxP = nullptr, *TyP = nullptr;
  T* TyR = nullptr;
};

template <typename T>
struct MGLevel {
  Geom g;
  Coef<T> c, cP;     // operator coefficients: V and D' blocks / pressure Laplacian
  LevelCoef<T> own;  // arrays owned by this hierarchy (FP32 copies), or empty
  Block<T> V, D, Pb;
};

template <typename T>
struct MG {
  std::vector<MGLevel<T>> L;
  double *AinvV = nullptr, *AinvD = nullptr, *AinvP = nullptr;
  int *idxV = nullptr, *idxD = nullptr, *idxP = nullptr;
  int mV = 0, mD = 0, mP = 0;  // unknowns of the coarsest V, D' and pressure-Laplacian blocks
  T* chtab = nullptr;  // Chebyshev coefficients, 16 per (level, block): a[0..7], c[8..15]
  int fuse_from = -1;  // first level handled by the fused single-CTA coarse cycle
  CoarseCycle<T> cycV, cycD, cycP;
};

// grids with at most this many cells per side run fused (measured: 16 beats 32, most in FP64)
const int FUSE_N = 16;
// levels up to this many cells per side take their residual and restriction
// inside the pre-smoothing tile (latency-bound launches there; on larger
// levels the wider halo it needs costs more than the two launches)
const int RR_MAX_N = 256;
const int SMALL_TILE_N = 256;  // levels up to this size smooth 4-row tiles (measured 1.4 % per step at 1024^2)

// the channel coarsens to at most this many cells per side (its coarsest
// dense velocity block has 6 n^2 + 4 n unknowns, 416 at 8)
const int CHANNEL_COARSEST_MAX = 8;

// the coarsening target of the options
int coarsest_of(const sd_options& o) {
  return o.geometry == SD_GEO_CHANNEL ? std::min(o.coarsest, CHANNEL_COARSEST_MAX) : o.coarsest;
}

int level_count(int n, int coarsest) {
  int L = 1;
  while (n % 2 == 0 && n / 2 >= 2 && n > coarsest) {
    n /= 2;
    ++L;
  }
  return L;
}

}  // namespace

struct sd_handle {
  std::mutex mtx;
  int n = 0;
  double mu = 1, alpha = 1, dt = 1;
  sd_options opt;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  cudaStream_t s2 = nullptr;                   // second stream (Darcy V-cycle overlap)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // one captured Arnoldi step per basis index, per solve mode (monolithic, and the
  // free-flow and porous-medium subdomain solves of the partitioned coupling)
  std::vector<cudaGraphExec_t> gexec[5];
  std::vector<long long> gcount[5];            // kernels in each captured step
  // graph option 2: a whole FGMRES solve per solve mode as one graph with
  // device-side loop control (built for one right-hand side and iterate)
  struct SolveGraph {
    cudaGraphExec_t ex = nullptr;
    const double* b = nullptr;
    const double* x = nullptr;
    long long pre = 0, post = 0;  // kernels outside the graph's loops
    bool bad = false;             // could not be built: step-by-step replay
  };
  SolveGraph sg[5];
  Geom g;
  int nlev = 1;
  int m = 30;
  long long lenA = 0;  // padded vector stride of the Krylov bases
  int nblk = 1;
  Arena ar;
  std::vector<Geom> geo;
  std::vector<double*> Klev;
  std::vector<LevelCoef<double>> c64;  // FP64 coefficients of every level
  MG<float> mg32;
  MG<double> mg64;
  double *stage = nullptr, *x = nullptr, *xm = nullptr, *b = nullptr, *B0 = nullptr, *B1 = nullptr;
  double* xmm = nullptr;  // x^{n-2} (extrapolate >= 2)
  double* x3 = nullptr;   // x^{n-3} (extrapolate 3)
  // the operator applied to the solved states, Y[i] = A x^{n-i} (i < ydepth =
  // extrapolate + 1; whole-system coupling only): the step's first residual
  // b - A x^0 then comes from their extrapolation (k_yhist, k_resid_hist)
  // instead of an FP64 operator application.  Every whole-system residual
  // launch stores its A x in Y[0], so a step's solve leaves A x^n there;
  // ylev: the valid entries Y[0 .. ylev-1] between steps (a user solve,
  // which also writes Y[0], clears them; sd_set_state and sd_set_history
  // recompute them with the operator's own arithmetic, so a resumed run is
  // bitwise the uninterrupted one).
  double* Y[4] = {nullptr, nullptr, nullptr, nullptr};
  int ydepth = 0, ylev = 0;
  double *V = nullptr, *Z = nullptr, *partial = nullptr, *scal = nullptr, *st = nullptr, *flag = nullptr;
  // partitioned coupling: subdomain right-hand side and the IQN-ILS state
  double* bsub = nullptr;
  IqnState iqn;
  double* hflag = nullptr;  // pinned
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double t = 0.0;
  long long step = 0;
  bool have_prev = false;  // x_m holds the state of the previous time level
  // per-block residuals of the last solve, queued for the caller's next
  // synchronisation (queue_block_residuals / finish_block_residuals)
  bool blk_pending = false;
  double blk_bnorm = 0.0;
  // solved time levels among x, x_m, x_mm, x3 (the initial condition is not
  // one: it need not lie on the discrete trajectory)
  int levels = 0;
  // kernel timing (sd_profile): event pairs around launches of one kernel class
  int prof_id = -1;
  std::vector<cudaEvent_t> prof_ev;
  std::vector<double> prof_bytes_pending, prof_flops_pending;
  int prof_used = 0;
  double prof_ms = 0.0, prof_bytes = 0.0, prof_flops = 0.0;
  long long prof_launches = 0;
  // scalar slots in scal[]
  // S_VSC + j: the scale of basis vector j of the whole-system solve, which
  // keeps its basis vectors unnormalised (arnoldi_orth)
  static const int S_H1 = 0, S_H2 = 32, S_N2 = 64, S_B2 = 65, S_BN = 66, S_N2B = 67, S_REO = 68, S_BLK = 69,
                   S_Y = 96, S_CTL = 128, S_VSC = 200, S_RH = 240;
};

namespace {

// unknowns of the handle's dense state vector
long long dof_of(const sd_handle* h) { return sd_dof_count_geometry(h->n, h->opt.geometry); }

// Lay out (or, with ar.plan == false, assign) every buffer of the handle.
template <typename T>
void take_coef(Arena& a, const Geom& g, LevelCoef<T>& C) {
  C.w = a.take<T>(g.nx + 1);
  C.rg = a.take<T>(g.nx + 1);
  C.Tx = a.take<T>((long long)g.n * g.P);
  C.Ty = a.take<T>((long long)(g.n + 1) * g.P);
  C.wP = a.take<T>(g.nx + 1);
  C.rgP = a.take<T>(g.nx + 1);
  C.TxP = a.take<T>((long long)g.n * g.P);
  C.TyP = a.take<T>((long long)(g.n + 1) * g.P);
}

template <typename T>
void take_block(Arena& a, long long len, Block<T>& B) {
  B.b = a.take<T>(len);
  B.x = a.take<T>(len);
  B.x2 = a.take<T>(len);
  B.d = a.take<T>(len);
  B.r = a.take<T>(len);
}

template <typename T>
void plan_mg(sd_handle* h, MG<T>& M, bool own_coef) {
  Arena& a = h->ar;
  M.L.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    MGLevel<T>& L = M.L[l];
    const Geom& g = h->geo[l];
    L.g = g;
    if (own_coef) take_coef<T>(a, g, L.own);
    take_block<T>(a, g.lenV, L.V);
    take_block<T>(a, g.lenD, L.D);
    take_block<T>(a, g.lenD, L.Pb);
  }
  const Geom& gc = h->geo[h->nlev - 1];
  M.mV = gc.n * (gc.nx + 1) + (gc.n + 1) * gc.nx;
  M.mD = gc.n * gc.n;
  M.mP = gc.n * gc.nx;
  M.AinvV = a.take<double>((long long)M.mV * M.mV);
  M.AinvD = a.take<double>((long long)M.mD * M.mD);
  M.AinvP = a.take<double>((long long)M.mP * M.mP);
  M.idxV = a.take<int>(M.mV);
  M.idxD = a.take<int>(M.mD);
  M.idxP = a.take<int>(M.mP);
  M.chtab = a.take<T>((long long)h->nlev * 3 * 16);
}

void plan_all(sd_handle* h) {
  Arena& a = h->ar;
  const int n = h->n;
  const long long nd = dof_of(h);
  h->stage = a.take<double>(nd > (long long)n * n ? nd : (long long)n * n);
  h->Klev.resize(h->nlev);
  h->c64.resize(h->nlev);
  for (int l = 0; l < h->nlev; ++l) {
    const Geom& g = h->geo[l];
    h->Klev[l] = a.take<double>((long long)g.n * g.P);
    take_coef<double>(a, g, h->c64[l]);
    h->c64[l].TyR = a.take<double>((long long)(g.n + 1) * g.P);
  }
  const long long len = h->g.len;
  h->x = a.take<double>(len);
  h->xm = a.take<double>(len);
  if (h->opt.extrapolate >= 2) h->xmm = a.take<double>(len);
  if (h->opt.extrapolate >= 3) h->x3 = a.take<double>(len);
  if (h->opt.coupling != SD_PARTITIONED) {
    h->ydepth = h->opt.extrapolate + 1;
    for (int i = 0; i < h->ydepth; ++i) h->Y[i] = a.take<double>(len);
  }
  h->b = a.take<double>(len);
  h->B0 = a.take<double>(len);
  h->B1 = a.take<double>(len);
  h->V = a.take<double>((long long)(h->m + 1) * h->lenA);
  h->Z = a.take<double>((long long)h->m * h->lenA);
  h->partial = a.take<double>(
      std::max((long long)h->nblk * 32, (long long)std::max(4, apply_dots_max()) * resid_norms_blocks(h->g.nx, n)));
  h->scal = a.take<double>(256);
  h->st = a.take<double>((long long)(h->m + 1) * h->m + 3 * h->m + 1);
  h->flag = a.take<double>(8);
  if (h->opt.coupling == SD_PARTITIONED) {
    const int n = h->n, qm = h->opt.coupling_columns;
    const long long ld = (n + 31) / 32 * 32;
    h->bsub = a.take<double>(len);
    IqnState& q = h->iqn;
    q.n = n;
    q.qmax = qm;
    q.omega0 = h->opt.coupling_omega;
    q.ld = ld;
    q.v = a.take<double>(ld);
    q.p_prev = a.take<double>(ld);
    q.vt_prev = a.take<double>(ld);
    q.r_prev = a.take<double>(ld);
    q.Vc = a.take<double>(ld * qm);
    q.Wc = a.take<double>(ld * qm);
    q.Q = a.take<double>(ld * qm);
    q.R = a.take<double>((long long)qm * qm);
    q.scal = a.take<double>(8);
    q.pG = a.take<double>(ld);
    q.vt = a.take<double>(ld);
  }
  if (h->opt.precision == SD_MIXED) plan_mg<float>(h, h->mg32, true);
  else plan_mg<double>(h, h->mg64, false);
}

// the operator's coefficients of level l (poisson: the pressure-Laplacian set)
Coef<double> coef64(sd_handle* h, int l, bool poisson = false) {
  const Geom& g = h->geo[l];
  LevelCoef<double>& C = h->c64[l];
  Coef<double> c;
  c.n = g.n; c.P = g.P; c.h = g.h; c.mu = h->mu; c.cm = g.h * g.h / h->dt;
  c.nx = g.nx; c.iw = g.iw; c.cx = poisson ? g.nx : g.n;
  c.lat = h->opt.bc != SD_BC_MMS;
  c.w = poisson ? C.wP : C.w;
  c.rg = poisson ? C.rgP : C.rg;
  c.Tx = poisson ? C.TxP : C.Tx;
  c.Ty = poisson ? C.TyP : C.Ty;
  finish_coef(c);
  return c;
}

// the coefficients the multigrid of block kind (0 V, 1 D', 2 pressure
// Laplacian) smooths with: the operator's, with the Darcy block's Ty replaced
// by TyR (the velocity block reads no Ty)
Coef<double> coef64_mg(sd_handle* h, int l, int kind) {
  Coef<double> c = coef64(h, l, kind == 2);
  if (kind != 2) c.Ty = h->c64[l].TyR;
  return c;
}

template <typename T>
void bind_coef(sd_handle* h, MG<T>& M) {
  for (int l = 0; l < h->nlev; ++l) {
    MGLevel<T>& L = M.L[l];
    const Geom& g = h->geo[l];
    L.c.n = g.n; L.c.P = g.P; L.c.h = (T)g.h; L.c.mu = (T)h->mu; L.c.cm = (T)(g.h * g.h / h->dt);
    L.c.nx = g.nx; L.c.iw = g.iw; L.c.cx = g.n;
    L.c.lat = h->opt.bc != SD_BC_MMS;
    L.cP = L.c;
    L.cP.cx = g.nx;
    L.c.w = L.own.w; L.c.rg = L.own.rg; L.c.Tx = L.own.Tx; L.c.Ty = L.own.Ty;
    L.cP.w = L.own.wP; L.cP.rg = L.own.rgP; L.cP.Tx = L.own.TxP; L.cP.Ty = L.own.TyP;
    finish_coef(L.c);
    finish_coef(L.cP);
  }
}
template <>
void bind_coef<double>(sd_handle* h, MG<double>& M) {
  for (int l = 0; l < h->nlev; ++l) {
    M.L[l].c = coef64_mg(h, l, 0);
    M.L[l].cP = coef64_mg(h, l, 2);
  }
}

// Chebyshev step coefficients on [lmax/ratio, 1.1 lmax] of D^-1 A.
template <typename T>
void cheb_coeffs(double lmax, double ratio, int deg, std::vector<T>& a, std::vector<T>& c) {
  const double hi = 1.1 * lmax, lo = lmax / ratio;
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  a.assign(deg, T(0));
  c.assign(deg, T(0));
  double rho = 1.0 / sigma;
  c[0] = (T)(1.0 / theta);
  for (int k = 1; k < deg; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    a[k] = (T)(rn * rho);
    c[k] = (T)(2.0 * rn / delta);
    rho = rn;
  }
}

// Largest eigenvalues of D^-1 A for every (level, block) of the hierarchy by
// FP64 power iteration (lam[3 l + kind], kind 0 V, 1 D', 2 pressure
// Laplacian; the coarsest level has none).  The chains run in rounds: one
// iteration of every unconverged chain is queued, then one read-back decides
// which go on, so a setup waits on the host once per round rather than once
// per iteration of every chain.  The chains of each block kind run on their
// own stream (s and two forked from it), with their own reduction scratch.
// Each chain has its own vectors (the Krylov bases are free during setup) and
// does the arithmetic of a chain run alone, in the same order.
int power_lmax_all(sd_handle* h, std::vector<double>& lam, cudaStream_t s) {
  struct Chain {
    int l, kind;
    long long len;
    Coef<double> c;
    double *x, *y;
    double lam;
    bool done;
  };
  const int nl = h->nlev - 1;
  lam.assign((size_t)3 * std::max(nl, 0), 0.0);
  std::vector<Chain> all;
  for (int l = 0; l < nl; ++l)
    for (int kind = 0; kind < 3; ++kind) {
      const Geom& g = h->geo[l];
      Chain ch;
      ch.l = l;
      ch.kind = kind;
      ch.len = kind == 0 ? g.lenV : g.lenD;
      ch.c = coef64_mg(h, l, kind);
      ch.x = ch.y = nullptr;
      ch.lam = 0.0;
      ch.done = false;
      all.push_back(ch);
    }
  // the Krylov bases V (m + 1 slots) and Z (m slots) as one pool of vectors;
  // the norms go to scal[0 .. 64) (no solve runs during setup)
  const long long vcap = (long long)(h->m + 1) * h->lenA, zcap = (long long)h->m * h->lenA;
  // stream k's dot partials go to partial + k nblk (partial holds 32 nblk doubles)
  cudaStream_t ks[3] = {s, nullptr, nullptr};
  cudaEvent_t kev[3] = {nullptr, nullptr, nullptr};
  int rc = SD_OK;
  for (int k = 0; k < 3 && rc == SD_OK; ++k)
    if (cudaEventCreateWithFlags(&kev[k], cudaEventDisableTiming) != cudaSuccess) rc = SD_E_CUDA;
  for (int k = 1; k < 3 && rc == SD_OK; ++k)
    if (cudaStreamCreateWithFlags(&ks[k], cudaStreamNonBlocking) != cudaSuccess) rc = SD_E_CUDA;
  if (rc == SD_OK && cudaEventRecord(kev[0], s) != cudaSuccess) rc = SD_E_CUDA;
  for (int k = 1; k < 3 && rc == SD_OK; ++k)
    if (cudaStreamWaitEvent(ks[k], kev[0], 0) != cudaSuccess) rc = SD_E_CUDA;
  auto join = [&]() {  // streams 1 and 2 into s
    for (int k = 1; k < 3; ++k)
      if (ks[k] && (cudaEventRecord(kev[k], ks[k]) != cudaSuccess || cudaStreamWaitEvent(s, kev[k], 0) != cudaSuccess))
        rc = SD_E_CUDA;
  };
  auto cleanup = [&]() {
    for (int k = 0; k < 3; ++k) {
      if (kev[k]) cudaEventDestroy(kev[k]);
      if (k > 0 && ks[k]) cudaStreamDestroy(ks[k]);
    }
  };
  if (rc != SD_OK) {
    join();
    cleanup();
    return rc;
  }
  size_t next = 0;
  while (next < all.size() && rc == SD_OK) {
    // as many chains as the two bases hold (each needs x and y; a chain of
    // the finest velocity block fits in V alone, whatever m)
    std::vector<Chain*> grp;
    long long vused = 0, zused = 0;
    while (next < all.size() && (int)grp.size() < 64) {
      const long long pad = (all[next].len + 31) / 32 * 32, need = 2 * pad;
      double* base = nullptr;
      if (vused + need <= vcap) {
        base = h->V + vused;
        vused += need;
      } else if (zused + need <= zcap) {
        base = h->Z + zused;
        zused += need;
      } else if (grp.empty()) {
        join();
        cleanup();
        return SD_E_NOMEM;
      } else {
        break;
      }
      Chain& ch = all[next++];
      ch.x = base;
      ch.y = base + pad;
      grp.push_back(&ch);
    }
    auto apply = [&](Chain& ch, const double* in, double* o) {
      if (ch.kind == 0) launch_resid_V<double>(ch.c, in, nullptr, o, 1, 1, 0, ks[0]);
      else launch_resid_D<double>(ch.c, in, nullptr, o, 1, 1, 0, ks[ch.kind]);
    };
    int q0 = 0;
    for (Chain* ch : grp) {
      cudaStream_t sk = ks[ch->kind];
      if (cudaMemsetAsync(ch->y, 0, sizeof(double) * ch->len, sk) != cudaSuccess) rc = SD_E_CUDA;
      launch_hash_fill(ch->x, ch->len, 1234u + (unsigned)ch->l, sk);
      apply(*ch, ch->x, ch->y);  // y has zero padding from here on
      launch_dot(ch->y, ch->y, ch->len, h->partial + (long long)ch->kind * h->nblk, reduce_blocks(ch->len),
                 h->scal + q0++, sk);
    }
    for (int it = 0; it < 25 && rc == SD_OK; ++it) {
      int q = 0;
      for (Chain* ch : grp) {
        const int slot = q++;
        if (ch->done) continue;
        const int nb = reduce_blocks(ch->len);
        cudaStream_t sk = ks[ch->kind];
        // the slot holds ||y||^2 of this y from the end of the previous
        // iteration (or the start): the same kernel on the same vector
        launch_scale_by(ch->y, ch->x, ch->len, h->scal + slot, 1, sk);
        apply(*ch, ch->x, ch->y);
        launch_dot(ch->y, ch->y, ch->len, h->partial + (long long)ch->kind * h->nblk, nb, h->scal + slot, sk);
      }
      join();
      std::vector<double> nrm(grp.size());
      if (cudaMemcpyAsync(nrm.data(), h->scal, sizeof(double) * grp.size(), cudaMemcpyDeviceToHost, s) !=
              cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        rc = SD_E_CUDA;
        break;
      }
      bool any = false;
      q = 0;
      for (Chain* ch : grp) {
        const double nv = std::sqrt(nrm[q++]);
        if (ch->done) continue;
        if (it > 4 && std::fabs(nv - ch->lam) <= 1e-3 * nv) ch->done = true;
        ch->lam = nv;
        any = any || !ch->done;
      }
      if (!any) break;
    }
    for (Chain* ch : grp) lam[(size_t)3 * ch->l + ch->kind] = ch->lam;
  }
  join();
  cleanup();
  return rc;
}

// Dense inverses of the coarsest V, D' and pressure-Laplacian blocks: apply
// the FP64 operator to unit vectors, gather the columns, invert by
// Gauss-Jordan on the device.  The three are independent and run
// concurrently on three streams, with one scratch allocation for all:
// coarse_inverses_begin queues them, coarse_inverses_end joins the streams,
// waits and checks the pivots.
struct InverseJob {
  double* scratch = nullptr;
  int* status = nullptr;
  cudaStream_t s3 = nullptr;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
  cudaStream_t st[3] = {nullptr, nullptr, nullptr};
  std::vector<int> idx[3];
  int rc = SD_OK;
};

template <typename T>
int coarse_inverses_begin(sd_handle* h, MG<T>& M, InverseJob& J) {
  const int l = h->nlev - 1;
  const Geom& g = h->geo[l];
  const int ms[3] = {M.mV, M.mD, M.mP};
  double* Ainv[3] = {M.AinvV, M.AinvD, M.AinvP};
  int* idxd[3] = {M.idxV, M.idxD, M.idxP};
  long long stride[3], off[3][4], tot = 0;
  for (int kind = 0; kind < 3; ++kind) {
    stride[kind] = kind == 0 ? g.lenV : g.lenD;
    const long long m = ms[kind];
    const long long sz[4] = {stride[kind] * m, stride[kind] * m, m * m, m};  // X, Y, A, fc (doubles)
    for (int q = 0; q < 4; ++q) {
      off[kind][q] = tot;
      tot += (sz[q] + 31) / 32 * 32;
    }
  }
  CK(cudaMalloc(&J.scratch, sizeof(double) * tot + 6 * sizeof(int)));
  double* scratch = J.scratch;
  int* status = J.status = reinterpret_cast<int*>(scratch + tot);  // three statuses, then three completion counters
  int& rc = J.rc;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == SD_OK) rc = SD_E_CUDA;
    return e == cudaSuccess;
  };
  ok(cudaStreamCreateWithFlags(&J.s3, cudaStreamNonBlocking));
  for (int q = 0; q < 3; ++q) ok(cudaEventCreateWithFlags(&J.ev[q], cudaEventDisableTiming));
  J.st[0] = h->s;
  J.st[1] = h->s2;
  J.st[2] = J.s3;
  const cudaStream_t* st = J.st;
  if (rc == SD_OK) {
    ok(cudaEventRecord(J.ev[0], h->s));
    ok(cudaStreamWaitEvent(h->s2, J.ev[0], 0));
    ok(cudaStreamWaitEvent(J.s3, J.ev[0], 0));
  }
  std::vector<int>* idx = J.idx;
  for (int kind = 0; kind < 3 && rc == SD_OK; ++kind) {
    const int m = ms[kind];
    const bool blockV = kind == 0;
    cudaStream_t s = st[kind];
    idx[kind].resize(m);
    int k = 0;
    if (blockV) {
      for (int j = 0; j < g.n; ++j)
        for (int i = 0; i <= g.nx; ++i) idx[kind][k++] = j * g.P + i;
      for (int j = 0; j <= g.n; ++j)
        for (int i = 0; i < g.nx; ++i) idx[kind][k++] = (int)(g.ov + (long long)j * g.P + i);
    } else {
      const int cx = kind == 2 ? g.nx : g.n;  // pressure Laplacian: the free-flow cells
      for (int j = 0; j < g.n; ++j)
        for (int i = 0; i < cx; ++i) idx[kind][k++] = j * g.P + i;
    }
    double* X = scratch + off[kind][0];
    double* Y = scratch + off[kind][1];
    double* A = scratch + off[kind][2];
    double* fc = scratch + off[kind][3];
    ok(cudaMemcpyAsync(idxd[kind], idx[kind].data(), sizeof(int) * m, cudaMemcpyHostToDevice, s));
    ok(cudaMemsetAsync(X, 0, sizeof(double) * stride[kind] * m, s));
    ok(cudaMemsetAsync(Y, 0, sizeof(double) * stride[kind] * m, s));
    launch_identity_batch(X, stride[kind], idxd[kind], m, s);
    Coef<double> c = coef64_mg(h, l, kind);
    if (blockV) launch_resid_V<double>(c, X, nullptr, Y, 2, m, stride[kind], s);
    else launch_resid_D<double>(c, X, nullptr, Y, 2, m, stride[kind], s);
    launch_gather_dense(Y, stride[kind], idxd[kind], m, A, s);
    launch_gj_inverse(A, Ainv[kind], m, fc, status + kind, status + 3 + kind, s);
  }
  return rc;
}

int coarse_inverses_end(sd_handle* h, InverseJob& J) {
  int& rc = J.rc;
  auto ok = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == SD_OK) rc = SD_E_CUDA;
    return e == cudaSuccess;
  };
  int hs[3] = {0, 0, 0};
  for (int q = 1; q < 3; ++q) {
    if (!J.st[q]) continue;
    ok(cudaEventRecord(J.ev[q], J.st[q]));
    ok(cudaStreamWaitEvent(h->s, J.ev[q], 0));
  }
  if (J.status) ok(cudaMemcpyAsync(hs, J.status, 3 * sizeof(int), cudaMemcpyDeviceToHost, h->s));
  ok(cudaStreamSynchronize(h->s));
  for (int q = 0; q < 3; ++q)
    if (J.ev[q]) cudaEventDestroy(J.ev[q]);
  if (J.s3) cudaStreamDestroy(J.s3);
  if (J.scratch) cudaFree(J.scratch);
  J = InverseJob();
  if (rc != SD_OK) return rc;
  for (int kind = 0; kind < 3; ++kind)
    if (hs[kind] != 0) {
      snprintf(g_errmsg, sizeof(g_errmsg), "coarsest %s block singular at column %d",
               kind == 0 ? "velocity" : (kind == 1 ? "Darcy" : "pressure-Laplacian"), hs[kind]);
      return SD_E_NUMERIC;
    }
  return SD_OK;
}

template <typename T>
int setup_mg(sd_handle* h, MG<T>& M) {
  cudaStream_t s = h->s;
  bind_coef<T>(h, M);
  for (int l = 0; l < h->nlev; ++l) {
    MGLevel<T>& L = M.L[l];
    if (!L.own.w) continue;
    const LevelCoef<double>& C = h->c64[l];
    const long long nx = (long long)L.g.n * L.g.P, ny = (long long)(L.g.n + 1) * L.g.P;
    launch_convert<T>(C.w, L.own.w, L.g.nx + 1, s);
    launch_convert<T>(C.rg, L.own.rg, L.g.nx + 1, s);
    launch_convert<T>(C.Tx, L.own.Tx, nx, s);
    launch_convert<T>(C.TyR, L.own.Ty, ny, s);
    launch_convert<T>(C.wP, L.own.wP, L.g.nx + 1, s);
    launch_convert<T>(C.rgP, L.own.rgP, L.g.nx + 1, s);
    launch_convert<T>(C.TxP, L.own.TxP, nx, s);
    launch_convert<T>(C.TyP, L.own.TyP, ny, s);
  }
  // the coarse inverses (three streams) and the power iterations (a fourth)
  // are independent: they run at the same time
  // (the power iterations' stream forks from s before the inverses are queued on it)
  cudaStream_t sp = nullptr;
  cudaEvent_t ef = nullptr;
  int rp = SD_OK;
  if (cudaStreamCreateWithFlags(&sp, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ef, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ef, s) != cudaSuccess ||
      cudaStreamWaitEvent(sp, ef, 0) != cudaSuccess)
    rp = SD_E_CUDA;
  InverseJob job;
  const int rb = coarse_inverses_begin<T>(h, M, job);
  std::vector<double> lams;
  if (rb == SD_OK && rp == SD_OK) {
    rp = power_lmax_all(h, lams, sp);
    if (cudaStreamSynchronize(sp) != cudaSuccess && rp == SD_OK) rp = SD_E_CUDA;
  }
  if (ef) cudaEventDestroy(ef);
  if (sp) cudaStreamDestroy(sp);
  const int re = coarse_inverses_end(h, job);
  CKR(rb);
  CKR(re);
  CKR(rp);
  const int deg = h->opt.cheb_degree;
  for (int l = 0; l + 1 < h->nlev; ++l) {
    const double lv = lams[(size_t)3 * l], ld = lams[(size_t)3 * l + 1], lp = lams[(size_t)3 * l + 2];
    const int dl = (l > 0 && h->opt.cheb_degree_coarse > 0) ? h->opt.cheb_degree_coarse : deg;
    const int dp = h->opt.schur_degree > 0 ? h->opt.schur_degree : dl;
    cheb_coeffs<T>(lv, h->opt.cheb_ratio, dl, M.L[l].V.cha, M.L[l].V.chc);
    cheb_coeffs<T>(ld, h->opt.cheb_ratio, dl, M.L[l].D.cha, M.L[l].D.chc);
    cheb_coeffs<T>(lp, h->opt.cheb_ratio, dp, M.L[l].Pb.cha, M.L[l].Pb.chc);
  }
  // the same coefficients in device memory: a lockstep batch reads each
  // instance's own (they differ with the spectrum of its operator)
  {
    std::vector<T> tab((size_t)h->nlev * 3 * 16, T(0));
    for (int l = 0; l + 1 < h->nlev; ++l) {
      Block<T>* bl[3] = {&M.L[l].V, &M.L[l].D, &M.L[l].Pb};
      for (int q = 0; q < 3; ++q) {
        T* row = tab.data() + ((size_t)l * 3 + q) * 16;
        for (int k = 0; k < (int)bl[q]->cha.size() && k < 8; ++k) {
          row[k] = bl[q]->cha[k];
          row[8 + k] = bl[q]->chc[k];
        }
        bl[q]->cht = M.chtab + ((size_t)l * 3 + q) * 16;
      }
    }
    CK(cudaMemcpyAsync(M.chtab, tab.data(), sizeof(T) * tab.size(), cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
  }
  M.fuse_from = -1;
  if (h->opt.fuse_coarse && h->g.iw == 0) {  // (the fused cycle serves the square geometry)
    auto fill = [&](CoarseCycle<T>& q, int kind, int which, int f) {
      std::memset(&q, 0, sizeof(q));
      q.nlev = h->nlev - f;
      q.kind = kind;
      for (int l = f; l < h->nlev; ++l) {
        MGLevel<T>& L = M.L[l];
        q.c[l - f] = which == 2 ? L.cP : L.c;
        Block<T>& B = which == 0 ? L.V : (which == 1 ? L.D : L.Pb);
        q.deg[l - f] = (int)B.cha.size();
        q.cht[l - f] = l + 1 < h->nlev ? B.cht : nullptr;
        for (int k = 0; k < (int)B.cha.size() && k < 8 && l + 1 < h->nlev; ++k) {
          q.cha[l - f][k] = B.cha[k];
          q.chc[l - f][k] = B.chc[k];
        }
      }
      Block<T>& B0 = which == 0 ? M.L[f].V : (which == 1 ? M.L[f].D : M.L[f].Pb);
      q.b_in = B0.b;
      q.x_out = B0.x;
      q.Ainv = which == 0 ? M.AinvV : (which == 1 ? M.AinvD : M.AinvP);
      q.idx = which == 0 ? M.idxV : (which == 1 ? M.idxD : M.idxP);
      q.m = which == 0 ? M.mV : (which == 1 ? M.mD : M.mP);
    };
    // the largest entry grid (at most FUSE_N cells per side) whose levels fit in shared memory
    for (int f = 0; f < h->nlev; ++f) {
      // a lone coarsest level runs the multi-CTA dense solve instead
      if (h->geo[f].n > FUSE_N || h->nlev - f > SD_CYC_MAXL || h->nlev - f < 2) continue;
      fill(M.cycV, 0, 0, f);
      fill(M.cycD, 1, 1, f);
      fill(M.cycP, 1, 2, f);
      if (coarse_cycle_smem(M.cycV) <= 200 * 1024 && coarse_cycle_smem(M.cycD) <= 200 * 1024) {
        M.fuse_from = f;
        break;
      }
    }
  }
  return SD_OK;
}

// ------------------------------------------------------ kernel timing
// Accumulate the elapsed time of the recorded event pairs (the stream has
// been synchronised by the caller, so every event has completed).
void prof_flush(sd_handle* h) {
  for (int k = 0; k + 1 < h->prof_used; k += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->prof_ev[k], h->prof_ev[k + 1]) == cudaSuccess) {
      h->prof_ms += ms;
      h->prof_bytes += h->prof_bytes_pending[k / 2];
      h->prof_flops += h->prof_flops_pending[k / 2];
      h->prof_launches += 1;
    }
  }
  h->prof_used = 0;
}

struct ProfScope {
  sd_handle* h;
  bool on;
  ProfScope(sd_handle* hh, int id, double bytes, double flops = 0.0) : h(hh), on(hh->prof_id == id) {
    if (!on) return;
    if (h->prof_used + 2 > (int)h->prof_ev.size()) {
      cudaStreamSynchronize(h->s);
      prof_flush(h);
    }
    h->prof_bytes_pending[h->prof_used / 2] = bytes;
    h->prof_flops_pending[h->prof_used / 2] = flops;
    cudaEventRecord(h->prof_ev[h->prof_used++], h->s);
  }
  ~ProfScope() {
    if (on) cudaEventRecord(h->prof_ev[h->prof_used++], h->s);
  }
};

// Algorithmic bytes of one launch (compulsory traffic, each array once):
//  fine velocity-block Chebyshev step: read x_in (if any), b, d (if a != 0);
//  write d and x_out, over the 2n(n+1) velocity faces.
// faces of the velocity block: u n x (nx+1), v (n+1) x nx
double faces_V(const Geom& g) { return (double)g.n * (g.nx + 1) + (double)g.nx * (g.n + 1); }
double cheb_bytes_V(const Geom& g, size_t es, bool has_x, bool has_d) {
  const double nv = faces_V(g);
  return nv * es * (1.0 + (has_x ? 1 : 0) + (has_d ? 1 : 0) + 2.0);
}
//  tiled velocity smoothing: read b (and x_in), write x_out over the faces
//  (the small coarse correction read by the post-smoothing is not counted)
double tile_bytes_V(const Geom& g, size_t es, bool has_x) {
  const double nv = faces_V(g);
  return nv * es * (has_x ? 3.0 : 2.0);
}
//  whole-system FP64 operator, algorithmic flops: one multiply-add per stored
//  matrix entry, nnz = 2 * 11 (u, v rows) + 4 (continuity) per free-flow
//  cell and 5 (Darcy) per pm cell minus the eliminated boundary couplings,
//  about 31 per cell of the square geometry.
double apply_flops(const Geom& g) {
  const double n = g.n;
  const double nnz = 26.0 * g.nx * n + 5.0 * n * n - 6.0 * n;
  return 2.0 * nnz;
}
//  whole-system FP64 operator: read x (every unknown), the transmissibilities
//  (2n(n+1)) and interface coefficients (2n), read b if residual, write y.
double apply_bytes(const Geom& g, bool resid) {
  const double nd = faces_V(g) + (double)g.nx * g.n + (double)g.n * g.n;
  return 8.0 * (nd * (resid ? 3 : 2) + 2.0 * g.n * (g.n + 1) + 2.0 * g.n);
}

// ----------------------------------------------------------- V-cycles
template <typename T>
ChebSteps<T> steps_of(const Block<T>& B, int rows, int wave) {
  ChebSteps<T> cs;
  std::memset(&cs, 0, sizeof(cs));
  cs.ns = (int)B.cha.size();
  cs.rows = rows;
  cs.wave = wave;
  for (int k = 0; k < cs.ns && k < 8; ++k) {
    cs.a[k] = B.cha[k];
    cs.c[k] = B.chc[k];
  }
  return cs;
}

// smoothing tile height of a level with n cells per side: the option, or by
// default 4 rows up to n = 256 (the coarse levels run a few CTAs each, whose
// latency shorter tiles cut), 8 up to n = 1024 (more CTAs in flight) and 16
// above (less halo)
int tile_rows_of(const sd_handle* h, int n) {
  if (h->opt.tile_rows) return h->opt.tile_rows;
  return n <= SMALL_TILE_N ? 4 : n <= 1024 ? 8 : 16;
}

// register-column tile height of a cell-block level (tile = 2; 0:
// shared-memory tiles on this level): 8 rows for tile_rows 8 or 16, else 4
// (fewer registers, more warps in flight).  Measured at 1024^2 (mixed, per
// launch): Darcy block, three steps, 16.8 us against 20.4 with 8-row shared-
// memory tiles; pressure Laplacian, one step, 11.4 against 13.4; at 512^2 the
// shared-memory tiles were faster (8.0 against 9.3), and for the velocity
// block at every size (1024^2: 30.1 against 48.7), so levels below
// SD_WAVE_MIN_N cells per side and the velocity block keep them.
#ifndef SD_WAVE_MIN_N
#define SD_WAVE_MIN_N 1024
#endif
int wave_rows_of(const sd_handle* h, int n) {
  if (h->opt.tile != 2 || n < SD_WAVE_MIN_N) return 0;
  if (h->opt.tile_rows) return h->opt.tile_rows >= 8 ? 8 : 4;
  return 4;
}

// tiled smoothing (all steps of one smoothing in one kernel) is used for the
// FP32 hierarchy with at most four Chebyshev steps
template <typename T>
bool use_tiles(const sd_handle* h, const Block<T>& B) {
  return std::is_same<T, float>::value && h->opt.tile && B.cha.size() >= 1 && B.cha.size() <= 4;
}

// Velocity block: Chebyshev pre-smoothing from zero, residual, transposed
// bilinear restriction, coarse correction, bilinear prolongation,
// Chebyshev post-smoothing; dense FP64 solve on the coarsest grid.
template <typename T>
void vcycle_V(MG<T>& M, int l, cudaStream_t s, sd_handle* prof_owner) {
  MGLevel<T>& L = M.L[l];
  Block<T>& B = L.V;
  if (l == M.fuse_from && launch_coarse_cycle<T>(M.cycV, s) == 0) {
    B.res = B.x;
    return;
  }
  if (l + 1 == (int)M.L.size()) {
    launch_dense_solve<T>(M.AinvV, M.idxV, M.mV, B.b, B.x, s);
    B.res = B.x;
    return;
  }
  MGLevel<T>& C = M.L[l + 1];
  T* cur = nullptr;
  const bool tiles = use_tiles(prof_owner, B);
  const int h_tile_rows = tile_rows_of(prof_owner, L.g.n), h_wave = 0;
  bool fused = false;  // residual and restriction taken by the pre-smoothing tile
  if (tiles) {
    ProfScope ps(prof_owner, l == 0 ? SD_PROF_CHEB_V : -2, tile_bytes_V(L.g, sizeof(T), false));
    if constexpr (std::is_same<T, float>::value) {
      const ChebSteps<T> cs = steps_of(B, h_tile_rows, h_wave);
      if (L.g.n <= RR_MAX_N)
        fused = launch_smooth_tile_V_rr<T>(L.c, B.b, B.x, cs, B.cht, C.g.n, C.g.P, C.V.b, s) == 0;
      if (!fused) launch_smooth_tile_V<T>(L.c, nullptr, B.b, B.x, cs, B.cht, nullptr, 0, 0, s);
    }
    cur = B.x;
  } else {
    for (int k = 0; k < (int)B.cha.size(); ++k) {
      T* out = (cur == B.x) ? B.x2 : B.x;
      {
        ProfScope ps(prof_owner, l == 0 ? SD_PROF_CHEB_V : -2, cheb_bytes_V(L.g, sizeof(T), cur != nullptr, k > 0));
        launch_cheb_V<T>(L.c, cur, B.b, B.d, out, B.cha[k], B.chc[k], B.cht ? B.cht + k : nullptr, 1, 0, s);
      }
      cur = out;
    }
  }
  if (!fused) {
    launch_resid_V<T>(L.c, cur, B.b, B.r, 0, 1, 0, s);
    launch_restrict_V<T>(L.g.n, L.g.P, B.r, C.g.n, C.g.nx, C.g.iw, C.g.P, C.V.b, L.c.lat, s);
  }
  vcycle_V(M, l + 1, s, prof_owner);
  if (tiles) {  // prolongation folded into the post-smoothing tile load
    T* out = (cur == B.x) ? B.x2 : B.x;
    ProfScope ps(prof_owner, l == 0 ? SD_PROF_CHEB_V : -2, tile_bytes_V(L.g, sizeof(T), true));
    if constexpr (std::is_same<T, float>::value)
      launch_smooth_tile_V<T>(L.c, cur, B.b, out, steps_of(B, h_tile_rows, h_wave), B.cht, C.V.res, C.g.n, C.g.P, s);
    cur = out;
  } else {
    launch_prolong_V<T>(L.g.n, L.g.P, cur, C.g.n, C.g.nx, C.g.iw, C.g.P, C.V.res, L.c.lat, s);
    for (int k = 0; k < (int)B.cha.size(); ++k) {
      T* out = (cur == B.x) ? B.x2 : B.x;
      {
        ProfScope ps(prof_owner, l == 0 ? SD_PROF_CHEB_V : -2, cheb_bytes_V(L.g, sizeof(T), true, k > 0));
        launch_cheb_V<T>(L.c, cur, B.b, B.d, out, B.cha[k], B.chc[k], B.cht ? B.cht + k : nullptr, 1, 0, s);
      }
      cur = out;
    }
  }
  B.res = cur;
}

// Cell-centred block (Darcy D' with its TPFA coefficients, or the pressure
// Laplacian P): same cycle with cell-sum restriction and bilinear prolongation.
template <typename T>
void vcycle_cell(MG<T>& M, int l, bool poisson, cudaStream_t s, const sd_handle* h) {
  MGLevel<T>& L = M.L[l];
  Block<T>& B = poisson ? L.Pb : L.D;
  const Coef<T>& c = poisson ? L.cP : L.c;
  if (l == M.fuse_from && launch_coarse_cycle<T>(poisson ? M.cycP : M.cycD, s) == 0) {
    B.res = B.x;
    return;
  }
  if (l + 1 == (int)M.L.size()) {
    launch_dense_solve<T>(poisson ? M.AinvP : M.AinvD, poisson ? M.idxP : M.idxD, poisson ? M.mP : M.mD, B.b, B.x, s);
    B.res = B.x;
    return;
  }
  MGLevel<T>& C = M.L[l + 1];
  Block<T>& BC = poisson ? C.Pb : C.D;
  T* cur = nullptr;
  const bool tiles = use_tiles(h, B);
  const int h_tile_rows = tile_rows_of(h, L.g.n), h_wave = wave_rows_of(h, L.g.n);
  bool fused = false;  // residual and restriction taken by the pre-smoothing tile
  if (tiles) {
    if constexpr (std::is_same<T, float>::value) {
      const ChebSteps<T> cs = steps_of(B, h_tile_rows, h_wave);
      if (L.g.n <= RR_MAX_N) fused = launch_smooth_tile_D_rr<T>(c, B.b, B.x, cs, B.cht, C.g.n, C.g.P, BC.b, s) == 0;
      if (!fused) launch_smooth_tile_D<T>(c, nullptr, B.b, B.x, cs, B.cht, nullptr, 0, 0, s);
    }
    cur = B.x;
  } else {
    for (int k = 0; k < (int)B.cha.size(); ++k) {
      T* out = (cur == B.x) ? B.x2 : B.x;
      launch_cheb_D<T>(c, cur, B.b, B.d, out, B.cha[k], B.chc[k], B.cht ? B.cht + k : nullptr, 1, 0, s);
      cur = out;
    }
  }
  if (!fused) launch_resid_restrict_D<T>(c, cur, B.b, C.g.n, C.g.P, BC.b, s);
  vcycle_cell(M, l + 1, poisson, s, h);
  if (tiles) {  // prolongation folded into the post-smoothing tile load
    T* out = (cur == B.x) ? B.x2 : B.x;
    if constexpr (std::is_same<T, float>::value)
      launch_smooth_tile_D<T>(c, cur, B.b, out, steps_of(B, h_tile_rows, h_wave), B.cht, BC.res, C.g.n, C.g.P, s);
    cur = out;
  } else {
    launch_prolong_D<T>(L.g.n, c.cx, L.g.P, cur, C.g.n, C.g.P, BC.res, s);
    for (int k = 0; k < (int)B.cha.size(); ++k) {
      T* out = (cur == B.x) ? B.x2 : B.x;
      launch_cheb_D<T>(c, cur, B.b, B.d, out, B.cha[k], B.chc[k], B.cht ? B.cht + k : nullptr, 1, 0, s);
      cur = out;
    }
  }
  B.res = cur;
}

// z = P^{-1} r (Sec. 4 block preconditioner, see include/sd.h).  For
// SD_TRI_SCHUR the ff pressure block uses S^-1 = (mu/(gamma h^2)) I +
// (1/dt) L_p^-1 (viscous and mass-dominated limits of B^T V^-1 B), with
// L_p = B^T B / h^2 solved by its own V-cycle.
// rs (may be null: 1): the device scale of r (an unnormalised basis vector)
template <typename T>
void precond(sd_handle* h, MG<T>& M, const double* r, double* z, const double* rs) {
  cudaStream_t s = h->s;
  const Coef<double> c = coef64(h, 0);
  const int mode = h->opt.precond;
  const bool tri = mode == SD_TRI_SCHUR;
  const double schur = tri ? h->mu / (h->opt.schur_gamma * h->g.h * h->g.h) : 1.0;
  if (tri && h->opt.darcy_coupled == 2) {
    // Darcy first (block lower-triangular in the order p_pm, p_ff -> v): the
    // Darcy and pressure-Laplacian cycles depend only on r and run
    // concurrently on two streams; the velocity cycle then sees B z_pff and
    // B'_1 z_pm
    cudaEventRecord(h->ev_fork, s);
    cudaStreamWaitEvent(h->s2, h->ev_fork, 0);
    launch_convert<T>(r + h->g.opm, M.L[0].D.b, h->g.lenD, h->s2, rs);
    vcycle_cell<T>(M, 0, false, h->s2, h);
    launch_precond_exit<T>(c, z, M.L[0].D.res, h->s2);
    cudaEventRecord(h->ev_join, h->s2);
    const T* eP = nullptr;
    if (h->opt.schur_mass) {
      launch_convert<T>(r + h->g.opf, M.L[0].Pb.b, h->g.lenD, s, rs);
      vcycle_cell<T>(M, 0, true, s, h);
      eP = M.L[0].Pb.res;
    }
    cudaStreamWaitEvent(s, h->ev_join, 0);
    launch_precond_entry<T>(c, r, z, schur, eP, 1.0 / h->dt, 1, 1, M.L[0].V.b, s, rs);
    vcycle_V<T>(M, 0, s, h);
    launch_precond_mid<T>(c, r, z, M.L[0].V.res, 0, (T*)nullptr, s, rs);
    return;
  }
  // block-diagonal Darcy part (no C'_1 coupling): its V-cycle runs on the
  // second stream, overlapping the pressure and velocity cycles
  const bool overlap = tri && h->opt.darcy_coupled == 0;
  if (overlap) {
    cudaEventRecord(h->ev_fork, s);
    cudaStreamWaitEvent(h->s2, h->ev_fork, 0);
    launch_convert<T>(r + h->g.opm, M.L[0].D.b, h->g.lenD, h->s2, rs);
    vcycle_cell<T>(M, 0, false, h->s2, h);
    launch_precond_exit<T>(c, z, M.L[0].D.res, h->s2);
    cudaEventRecord(h->ev_join, h->s2);
  }
  const T* eP = nullptr;
  if (tri && h->opt.schur_mass) {
    launch_convert<T>(r + h->g.opf, M.L[0].Pb.b, h->g.lenD, s, rs);
    vcycle_cell<T>(M, 0, true, s, h);
    eP = M.L[0].Pb.res;
  }
  launch_precond_entry<T>(c, r, z, schur, eP, 1.0 / h->dt, tri, 0, M.L[0].V.b, s, rs);
  vcycle_V<T>(M, 0, s, h);
  if (mode == SD_PV_BGS_I) launch_precond_bgs_pff<T>(c, r, z, M.L[0].V.res, s, rs);
  if (overlap) {
    launch_precond_mid<T>(c, r, z, M.L[0].V.res, 0, (T*)nullptr, s, rs);
    cudaStreamWaitEvent(s, h->ev_join, 0);
    return;
  }
  launch_precond_mid<T>(c, r, z, M.L[0].V.res, mode != SD_PV_BJ_I, M.L[0].D.b, s, rs);
  vcycle_cell<T>(M, 0, false, s, h);
  launch_precond_exit<T>(c, z, M.L[0].D.res, s);
}

void apply_precond(sd_handle* h, const double* r, double* z, const double* rs = nullptr) {
  if (h->opt.precision == SD_MIXED) precond<float>(h, h->mg32, r, z, rs);
  else precond<double>(h, h->mg64, r, z, rs);
}

// ------------------------------------------------ solve modes
// FGMRES runs on the whole system (MODE_MONO) or, for the partitioned
// coupling, on one subdomain's rows of Eq. (9) with the other subdomain's
// unknowns held fixed: MODE_FF on the prefix [u | v | p_ff] of the
// whole-system layout, MODE_PM on the suffix p_pm.  Vectors keep the
// whole-system layout; a mode reads and writes only its own range.
// The order of Sec. 3 (free flow first) uses MODE_FFD, the free-flow rows
// with the interface velocity prescribed, and MODE_PMD, the Darcy rows with
// the interface pressure prescribed over the half cell below Gamma.
enum { MODE_MONO = 0, MODE_FF = 1, MODE_PM = 2, MODE_FFD = 3, MODE_PMD = 4 };

struct Range {
  long long off, len;
};
Range mode_range(const sd_handle* h, int mode) {
  if (mode == MODE_FF || mode == MODE_FFD) return {0, h->g.opm};
  if (mode == MODE_PM || mode == MODE_PMD) return {h->g.opm, h->g.lenD};
  return {0, h->g.len};
}

// Relative tolerance of a solve: rtol for the whole system; for a subdomain
// solve of the partitioned coupling, coupling_rtol, or, when that is 0,
// three decades below the relative change the coupling test resolves (not
// below 1e-12, near the FP64 floor of the solves, nor above rtol).
double mode_rtol(const sd_handle* h, int mode) {
  if (mode == MODE_MONO) return h->opt.rtol;
  if (h->opt.coupling_rtol > 0) return h->opt.coupling_rtol;
  return std::min(h->opt.rtol, std::max(1e-3 * h->opt.coupling_eps, 1e-12));
}
// A subdomain solve whose restart cycle did not halve the true residual has
// reached the rounding floor of its rows (which the tight tolerance above can
// lie below, e.g. Darcy rows whose right-hand side is only the small interface
// flux): it stops there, converged if its residual meets rtol (or its own
// tolerance, when looser), else SD_E_NOCONV.  0: never (whole system).
double mode_accept(const sd_handle* h, int mode) {
  if (mode == MODE_MONO) return 0.0;
  return std::max(h->opt.rtol, mode_rtol(h, mode));
}

// y = A_mode x, or y = b - A_mode x
void apply_op(sd_handle* h, int mode, const double* x, const double* b, double* y) {
  const Coef<double> c = coef64(h, 0);
  if (mode == MODE_FF || mode == MODE_FFD) {
    launch_apply_ff(c, x, b, y, mode == MODE_FFD, h->s);
  } else if (mode == MODE_PM) {
    const long long o = h->g.opm;
    launch_resid_D<double>(c, x + o, b ? b + o : nullptr, y + o, b ? 0 : 2, 1, 0, h->s);
  } else if (mode == MODE_PMD) {
    const long long o = h->g.opm;
    launch_apply_pmd(c, x + o, b ? b + o : nullptr, y + o, h->s);
  } else {
    launch_apply_full(c, x, b, y, h->s);
  }
}

// V_0 = b - A x and ||V_0||^2 into scal[S_B2] (with with_b also ||b||^2 into
// scal[S_BN]).  For the whole system the residual kernel forms the norms
// itself, together with the per-block norms scal[S_BLK + 0..2] (velocity,
// continuity and Darcy rows) that the step reports, so no separate dot
// products run.
void resid_norms(sd_handle* h, int mode, const double* x, const double* b, bool with_b) {
  double* sc = h->scal;
  if (mode == MODE_MONO) {
    launch_resid_norms(coef64(h, 0), x, b, h->V, h->partial, sc, sd_handle::S_BLK, sd_handle::S_B2,
                       sd_handle::S_BN, with_b ? 1 : 0, h->s, with_b && h->ydepth ? sd_handle::S_RH : -1,
                       h->ydepth ? h->Y[0] : nullptr);
    return;
  }
  const Range rg = mode_range(h, mode);
  const long long len = rg.len, o = rg.off;
  const int nb = reduce_blocks(len);
  if (with_b) launch_dot(b + o, b + o, len, h->partial, nb, sc + sd_handle::S_BN, h->s);
  apply_op(h, mode, x, b, h->V);
  launch_dot(h->V + o, h->V + o, len, h->partial, nb, sc + sd_handle::S_B2, h->s);
}

// Subdomain preconditioners: the free-flow part of the block preconditioner
// (Schur block and velocity V-cycle, no Darcy block) and the D' V-cycle.
template <typename T>
void precond_sub(sd_handle* h, MG<T>& M, int mode, const double* r, double* z) {
  cudaStream_t s = h->s;
  const Coef<double> c = coef64(h, 0);
  if (mode == MODE_PM || mode == MODE_PMD) {
    launch_convert<T>(r + h->g.opm, M.L[0].D.b, h->g.lenD, s);
    vcycle_cell<T>(M, 0, false, s, h);
    launch_precond_exit<T>(c, z, M.L[0].D.res, s);
    return;
  }
  const int pmode = h->opt.precond;
  const bool tri = pmode == SD_TRI_SCHUR;
  const double schur = tri ? h->mu / (h->opt.schur_gamma * h->g.h * h->g.h) : 1.0;
  const T* eP = nullptr;
  if (tri && h->opt.schur_mass) {
    launch_convert<T>(r + h->g.opf, M.L[0].Pb.b, h->g.lenD, s);
    vcycle_cell<T>(M, 0, true, s, h);
    eP = M.L[0].Pb.res;
  }
  launch_precond_entry<T>(c, r, z, schur, eP, 1.0 / h->dt, tri, 0, M.L[0].V.b, s);
  vcycle_V<T>(M, 0, s, h);
  if (pmode == SD_PV_BGS_I) launch_precond_bgs_pff<T>(c, r, z, M.L[0].V.res, s);
  launch_precond_mid<T>(c, r, z, M.L[0].V.res, 0, (T*)nullptr, s);
  if (mode == MODE_FFD)  // identity rows of the prescribed interface velocity
    cudaMemcpyAsync(z + h->g.ov, r + h->g.ov, sizeof(double) * h->n, cudaMemcpyDeviceToDevice, s);
}

void apply_precond_mode(sd_handle* h, int mode, const double* r, double* z, const double* rs = nullptr) {
  if (mode == MODE_MONO) {
    apply_precond(h, r, z, rs);
  } else if (h->opt.precision == SD_MIXED) {
    precond_sub<float>(h, h->mg32, mode, r, z);
  } else {
    precond_sub<double>(h, h->mg64, mode, r, z);
  }
}

// ----------------------------------------------------------- Arnoldi step
// z_j = P^-1 v_j, w = A z_j, then w orthogonalised against v_0..v_j and the
// new Hessenberg column rotated (Givens).  Orthogonalisation:
//   orth 0: classical Gram-Schmidt with one re-orthogonalisation (CGS2);
//   orth 1: the second pass only when the first removed nearly all of w
//           (||w'|| < eta ||w||, decided on the device).
void arnoldi_orth(sd_handle* h, int j, const double* vj, double* zj, double* w, int mode = MODE_MONO) {
  cudaStream_t s = h->s;
  const Range rg = mode_range(h, mode);
  const long long len = rg.len, vs = h->lenA;
  const int nb = reduce_blocks(len), m = h->m, k = j + 1;
  double* sc = h->scal;
  // the whole system keeps its basis vectors unnormalised: V_q stands for
  // vsc[q] W_q, the stored W_q being the Gram-Schmidt remainder w' (or the
  // residual for q = 0) and vsc[q] = 1 / ||W_q|| its scale (k_init_cycle,
  // k_givens); the scales enter the preconditioner's input (in FP64, before
  // its conversion: the same values as a normalised vector), the dots (after
  // their sums) and the updates' coefficients, so no pass over HBM
  // normalises a vector.  The subdomain solves normalise explicitly.
  const bool mono = mode == MODE_MONO;
  double* vsc = mono ? sc + sd_handle::S_VSC : nullptr;
  // the whole system's operator forms the first pass's dot products itself
  // (up to apply_dots_max() basis vectors): no second read of w for them
  const bool fused = mono && k <= apply_dots_max();
  apply_precond_mode(h, mode, vj, zj, mono ? vsc + j : nullptr);
  {
    const double dof = (double)dof_of(h);
    ProfScope ps(h, mono ? SD_PROF_APPLY : -2, apply_bytes(h->g, false) + (fused ? 8.0 * k * dof : 0.0),
                 apply_flops(h->g) + (fused ? 2.0 * k * dof : 0.0));
    if (fused) launch_apply_dots(coef64(h, 0), zj, w, h->V, vs, k, h->partial, s);
    else apply_op(h, mode, zj, nullptr, w);
  }
  const double* Vb = h->V + rg.off;
  w += rg.off;
  if (fused) {
    const int na = (int)resid_norms_blocks(h->g.nx, h->n);
    launch_reduce(h->partial, na, k, na, sc + sd_handle::S_H1, nullptr, s, vsc);
  } else {
    {
      ProfScope ps(h, SD_PROF_MDOT, 8.0 * (k + 1) * (double)len, 2.0 * k * (double)len);
      launch_mdot(Vb, vs, k, w, len, h->partial, nb, nb, nullptr, s);
    }
    launch_reduce(h->partial, nb, k, nb, sc + sd_handle::S_H1, nullptr, s, vsc);
  }
  if (h->opt.orth == 0) {
    {
      ProfScope ps(h, SD_PROF_MUPDATE, 8.0 * (k + 2) * (double)len, 4.0 * k * (double)len);
      launch_mupdate(Vb, vs, k, sc + sd_handle::S_H1, w, len, h->partial, nb, nb, 1, nullptr, s, vsc);
    }
    launch_reduce(h->partial, nb, k, nb, sc + sd_handle::S_H2, nullptr, s, vsc);
    {
      ProfScope ps(h, SD_PROF_MUPDATE, 8.0 * (k + 2) * (double)len, 2.0 * (k + 1) * (double)len);
      launch_mupdate(Vb, vs, k, sc + sd_handle::S_H2, w, len, h->partial, nb, nb, 2, nullptr, s, vsc);
    }
    launch_reduce(h->partial, nb, 1, nb, sc + sd_handle::S_N2B, nullptr, s);
    launch_givens(h->st, j, m, sc + sd_handle::S_H1, sc + sd_handle::S_H2, sc + sd_handle::S_N2,
                  sc + sd_handle::S_N2B, nullptr, h->flag, s, vsc);
  } else {
    double* reo = sc + sd_handle::S_REO;
    const double eta = h->opt.reorth_eta;
    {
      ProfScope ps(h, SD_PROF_MUPDATE, 8.0 * (k + 2) * (double)len, 2.0 * (k + 1) * (double)len);
      launch_mupdate(Vb, vs, k, sc + sd_handle::S_H1, w, len, h->partial, nb, nb, 2, nullptr, s, vsc);
    }
    launch_reduce_decide(h->partial, nb, sc + sd_handle::S_N2, sc + sd_handle::S_H1, k, eta * eta, reo, s);
    // the second pass: its launches return at once unless the decision asked for it
    launch_mdot(Vb, vs, k, w, len, h->partial, nb, nb, reo, s);
    launch_reduce(h->partial, nb, k, nb, sc + sd_handle::S_H2, reo, s, vsc);
    launch_mupdate(Vb, vs, k, sc + sd_handle::S_H2, w, len, h->partial, nb, nb, 2, reo, s, vsc);
    launch_reduce(h->partial, nb, 1, nb, sc + sd_handle::S_N2B, reo, s);
    launch_givens(h->st, j, m, sc + sd_handle::S_H1, sc + sd_handle::S_H2, sc + sd_handle::S_N2,
                  sc + sd_handle::S_N2B, reo, h->flag, s, vsc);
  }
  // the subdomain solves' new basis vector: w / h_{j+1,j}
  if (!mono) launch_scale_by(w, w, len, h->flag + 1, 0, s);
}

// Per-block residual norms of the whole-system residual r (in h->V, whole
// layout): the velocity rows [u | v], the continuity rows p_ff and the Darcy
// rows p_pm, each relative to ||b||.  Batched in a lockstep batch (t_bat).
void block_residual_dots(sd_handle* h) {
  const Geom& g = h->g;
  const long long lo[3] = {0, g.opf, g.opm}, hi[3] = {g.opf, g.opm, g.len};
  for (int q = 0; q < 3; ++q)
    launch_dot(h->V + lo[q], h->V + lo[q], hi[q] - lo[q], h->partial, reduce_blocks(hi[q] - lo[q]),
               h->scal + sd_handle::S_BLK + q, h->s);
}
int block_residuals(sd_handle* h, double bnorm, sd_step_info* info) {
  block_residual_dots(h);
  CK(cudaMemcpyAsync(h->hflag + 12, h->scal + sd_handle::S_BLK, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  CK(cudaStreamSynchronize(h->s));
  const double d = bnorm > 0 ? bnorm : 1.0;
  info->relres_v = std::sqrt(h->hflag[12]) / d;
  info->relres_pff = std::sqrt(h->hflag[13]) / d;
  info->relres_pm = std::sqrt(h->hflag[14]) / d;
  return SD_OK;
}

// The same without waiting: the dots and their copy are queued, and
// finish_block_residuals fills them in after the caller's next
// synchronisation of the stream (one host wait less per step).
int queue_block_residuals(sd_handle* h, double bnorm) {
  // the last whole-system residual (resid_norms) left them in S_BLK
  CK(cudaMemcpyAsync(h->hflag + 12, h->scal + sd_handle::S_BLK, 3 * sizeof(double), cudaMemcpyDeviceToHost, h->s));
  h->blk_pending = true;
  h->blk_bnorm = bnorm;
  return SD_OK;
}
void finish_block_residuals(sd_handle* h, sd_step_info* info) {
  if (!h->blk_pending) return;
  h->blk_pending = false;
  const double d = h->blk_bnorm > 0 ? h->blk_bnorm : 1.0;
  info->relres_v = std::sqrt(h->hflag[12]) / d;
  info->relres_pff = std::sqrt(h->hflag[13]) / d;
  info->relres_pm = std::sqrt(h->hflag[14]) / d;
}

// ------------------------------------------------- FGMRES as one graph
// Graph option 2: fgmres() below as one CUDA graph per solve mode, its
// decisions taken on the device.  Top level: ||b||, the first true residual
// and k_restart_ctrl, then a WHILE node over restart cycles, then (whole
// system) the per-block residual dots.  WHILE body: k_cycle_head, the cycle
// set-up, Arnoldi step 0 and k_step_ctrl, a chain of IF nodes for steps
// 1..m-1 (each body: the step and its k_step_ctrl, which sets the next IF's
// condition), then the update of x with k read on the device, the new true
// residual and k_restart_ctrl, which sets the WHILE condition.  The kernels
// and their order are those of the step-by-step path, so both give the same
// iterates bit for bit; the host waits once per solve instead of once per
// iteration.
int build_solve_graph(sd_handle* h, int mode, const double* b, double* x) {
  cudaStream_t s = h->s;
  const Range rg = mode_range(h, mode);
  const long long len = rg.len, vs = h->lenA, o = rg.off;
  const int m = h->m, nb = reduce_blocks(len), maxit = h->opt.max_iters;
  double* sc = h->scal;
  double* ctl = sc + sd_handle::S_CTL;
  const int pdl = t_pdl;
  const long long l_start = t_launch_count;
  cudaGraph_t top = nullptr;
  cudaGraphExec_t ex = nullptr;
  std::vector<cudaGraphNode_t> deps;
  bool capturing = false;
  long long pre = 0, post = 0;
  cudaError_t err = cudaSuccess;
  // capture into graph g after the nodes in deps (none if !after)
  auto begin = [&](cudaGraph_t g, bool after) {
    if (err != cudaSuccess) return false;
    err = cudaStreamBeginCaptureToGraph(s, g, after ? deps.data() : nullptr, nullptr, after ? deps.size() : 0,
                                        cudaStreamCaptureModeThreadLocal);
    capturing = err == cudaSuccess;
    return capturing;
  };
  // end the capture; keep: deps = its last nodes
  auto end = [&](bool keep) {
    if (!capturing) return;
    if (keep && err == cudaSuccess) {
      cudaStreamCaptureStatus cs;
      const cudaGraphNode_t* d = nullptr;
      size_t nd = 0;
      err = cudaStreamGetCaptureInfo(s, &cs, nullptr, nullptr, &d, nullptr, &nd);
      if (err == cudaSuccess) deps.assign(d, d + nd);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    capturing = false;
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = cudaGetLastError();
  };
  // conditional node of graph g after deps; its body in *body
  auto cond = [&](cudaGraph_t g, cudaGraphConditionalHandle hd, cudaGraphConditionalNodeType type,
                  cudaGraph_t* body) {
    if (err != cudaSuccess) return;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hd;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t nd = nullptr;
    err = cudaGraphAddNode(&nd, g, deps.data(), nullptr, deps.size(), &np);
    if (err != cudaSuccess) return;
    *body = np.conditional.phGraph_out[0];
    deps.assign(1, nd);
  };
  auto step = [&](int j) {
    const long long l0 = t_launch_count;
    double* vj = h->V + (long long)j * vs;
    double* zj = h->Z + (long long)j * vs;
    double* w = h->V + (long long)(j + 1) * vs;
    arnoldi_orth(h, j, vj, zj, w, mode);
    return t_launch_count - l0;
  };
  err = cudaGraphCreate(&top, 0);
  cudaGraphConditionalHandle loop = 0;
  CondSet cs = {};
  cs.n = m;
  if (err == cudaSuccess) err = cudaGraphConditionalHandleCreate(&loop, top, 0, cudaGraphCondAssignDefault);
  for (int j = 1; j < m && err == cudaSuccess; ++j)
    err = cudaGraphConditionalHandleCreate(&cs.c[j], top, 0, cudaGraphCondAssignDefault);
  // ||b||, the first true residual, and whether a cycle runs
  if (begin(top, false)) {
    const long long l0 = t_launch_count;
    resid_norms(h, mode, x, b, true);
    launch_solve_begin(sc + sd_handle::S_BN, mode_rtol(h, mode), mode_accept(h, mode), ctl, s);
    launch_restart_ctrl(sc + sd_handle::S_B2, ctl, maxit, 0.0, loop, s);
    pre = t_launch_count - l0;
    end(true);
  }
  cudaGraph_t wbody = nullptr;
  cond(top, loop, cudaGraphCondTypeWhile, &wbody);
  const std::vector<cudaGraphNode_t> after_loop = deps;
  // one restart cycle: set-up and Arnoldi step 0
  deps.clear();
  if (begin(wbody, false)) {
    const long long l0 = t_launch_count;
    launch_cycle_head(cs, s);
    launch_init_cycle(h->st, m, sc + sd_handle::S_B2, h->flag, s, sc + sd_handle::S_VSC);
    if (mode != MODE_MONO) launch_scale_by(h->V + o, h->V + o, len, h->flag + 1, 0, s);
    step(0);
    const long long k = t_launch_count - l0 + 1;
    launch_step_ctrl(h->flag, ctl, maxit, (double)k, m > 1, m > 1 ? cs.c[1] : 0, s);
    end(true);
  }
  for (int j = 1; j < m; ++j) {
    cudaGraph_t ib = nullptr;
    cond(wbody, cs.c[j], cudaGraphCondTypeIf, &ib);
    const std::vector<cudaGraphNode_t> keep = deps;
    if (begin(ib, false)) {
      const long long k = step(j) + 1;
      launch_step_ctrl(h->flag, ctl, maxit, (double)k, j + 1 < m, j + 1 < m ? cs.c[j + 1] : 0, s);
      end(false);
    }
    deps = keep;
  }
  // update of x with the cycle's k (flag[5]), the new true residual, and
  // whether another cycle runs; no programmatic edge out of a conditional node
  if (begin(wbody, true)) {
    const long long l0 = t_launch_count;
    t_pdl = 0;
    launch_backsolve(h->st, m, m, sc + sd_handle::S_Y, h->flag + 5, s);
    t_pdl = pdl;
    launch_axpy_multi(x + o, h->Z + o, vs, sc + sd_handle::S_Y, m, len, h->flag + 5, s);
    resid_norms(h, mode, x, b, false);
    const long long k = t_launch_count - l0 + 1;
    launch_restart_ctrl(sc + sd_handle::S_B2, ctl, maxit, (double)k, loop, s);
    end(false);
  }
  // (the per-block residual norms of the whole system are left in S_BLK by
  // the last residual inside the loop)
  t_pdl = pdl;
  if (capturing) end(false);
  if (err == cudaSuccess) err = cudaGraphInstantiate(&ex, top, 0);
  if (top) cudaGraphDestroy(top);
  // the capture went through the counting launch wrappers; replays are
  // credited from the graph's own counts
  g_launch_count.fetch_sub(t_launch_count - l_start);
  sd_handle::SolveGraph& G = h->sg[mode];
  if (err != cudaSuccess) {
    if (ex) cudaGraphExecDestroy(ex);
    cudaGetLastError();
    G.bad = true;
    return SD_E_CUDA;
  }
  G.ex = ex;
  G.b = b;
  G.x = x;
  G.pre = pre;
  G.post = post;
  return SD_OK;
}

// One FGMRES solve from the solve graph (see build_solve_graph); returns
// kNoGraph when the graph cannot be built, and the caller takes the
// step-by-step path.
constexpr int kNoGraph = 1;
int fgmres_graph(sd_handle* h, const double* b, double* x, sd_step_info* info, int mode) {
  cudaStream_t s = h->s;
  sd_handle::SolveGraph& G = h->sg[mode];
  if (G.ex && (G.b != b || G.x != x)) {
    CK(cudaStreamSynchronize(s));
    cudaGraphExecDestroy(G.ex);
    G.ex = nullptr;
  }
  if (!G.ex && build_solve_graph(h, mode, b, x) != SD_OK) return kNoGraph;
  CK(cudaGraphLaunch(G.ex, s));
  double* hc = h->hflag + 16;
  CK(cudaMemcpyAsync(hc, h->scal + sd_handle::S_CTL, C_COUNT * sizeof(double), cudaMemcpyDeviceToHost, s));
  if (mode == MODE_MONO)
    CK(cudaMemcpyAsync(h->hflag + 12, h->scal + sd_handle::S_BLK, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  g_launch_count.fetch_add(G.pre + G.post + (long long)hc[C_KERN]);
  const int status = hc[C_STAT] == C_STAT_NUMERIC ? SD_E_NUMERIC : hc[C_STAT] == C_STAT_NOCONV ? SD_E_NOCONV : SD_OK;
  if (info) {
    info->iters = (int)hc[C_ITER];
    info->restarts = (int)hc[C_REST];
    info->relres = hc[C_REL];
    info->status = status;
    info->reorths = (int)hc[C_REO];
    info->relres_v = info->relres_pff = info->relres_pm = -1.0;
    if (mode == MODE_MONO && status != SD_E_NUMERIC) {
      const double d = hc[C_BN] > 0 ? hc[C_BN] : 1.0;
      info->relres_v = std::sqrt(h->hflag[12]) / d;
      info->relres_pff = std::sqrt(h->hflag[13]) / d;
      info->relres_pm = std::sqrt(h->hflag[14]) / d;
    }
  }
  return status;
}

// --------------------------------------------------------------- FGMRES
// Flexible GMRES(m) with CGS2 orthogonalisation, all FP64.  x holds the
// initial guess.  The stopping test is the FP64 true residual
// ||b - A x||_2 <= rtol ||b||_2, checked at every restart and at the end.
int fgmres(sd_handle* h, const double* b, double* x, sd_step_info* info, int mode = MODE_MONO) {
  cudaStream_t s = h->s;
  if (h->opt.graph == 2 && h->prof_id < 0 && h->s != nullptr && !h->sg[mode].bad) {
    const int rc = fgmres_graph(h, b, x, info, mode);
    if (rc != kNoGraph) return rc;
  }
  const Range rg = mode_range(h, mode);
  const long long len = rg.len, vs = h->lenA, o = rg.off;
  const int m = h->m, nb = reduce_blocks(len);
  double* sc = h->scal;
  // ||b|| and the first true residual V_0 = b - A x, read back together (S_B2
  // and S_BN are adjacent slots)
  resid_norms(h, mode, x, b, true);
  CK(cudaMemcpyAsync(h->hflag + 5, sc + sd_handle::S_B2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const double bnorm = std::sqrt(h->hflag[6]);
  const double tol = mode_rtol(h, mode) * (bnorm > 0 ? bnorm : 1.0);
  const double acc = mode_accept(h, mode);
  const double acc_tol = acc > 0 ? acc * (bnorm > 0 ? bnorm : 1.0) : -1.0;
  int iters = 0, restarts = 0, status = SD_OK, reorths = 0;
  double relres = 0.0, prev = 0.0;
  bool first = true;
  for (;;) {
    if (!first) {
      resid_norms(h, mode, x, b, false);  // V_0 = b - A x
      CK(cudaMemcpyAsync(h->hflag + 5, sc + sd_handle::S_B2, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
    }
    first = false;
    const double beta = std::sqrt(h->hflag[5]);
    const double beta_prev = prev;
    prev = beta;
    relres = bnorm > 0 ? beta / bnorm : beta;
    if (!std::isfinite(beta)) { status = SD_E_NUMERIC; break; }
    if (beta <= tol) break;
    if (acc_tol >= 0.0 && restarts > 0 && beta > 0.5 * beta_prev) {  // stagnated (mode_accept)
      if (beta > acc_tol) status = SD_E_NOCONV;
      break;
    }
    if (iters >= h->opt.max_iters) { status = SD_E_NOCONV; break; }
    ++restarts;
    launch_init_cycle(h->st, m, sc + sd_handle::S_B2, h->flag, s, sc + sd_handle::S_VSC);
    if (mode != MODE_MONO) launch_scale_by(h->V + o, h->V + o, len, h->flag + 1, 0, s);
    int k = 0;
    bool numeric = false;
    for (int j = 0; j < m; ++j) {
      double* vj = h->V + (long long)j * vs;
      double* zj = h->Z + (long long)j * vs;
      double* w = h->V + (long long)(j + 1) * vs;
      std::vector<cudaGraphExec_t>& gx = h->gexec[mode];
      std::vector<long long>& gc = h->gcount[mode];
      if (h->opt.graph && h->prof_id < 0 && h->s != nullptr) {
        if (!gx[j]) {
          cudaGraph_t gr = nullptr;
          const long long l0 = t_launch_count;
          CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          arnoldi_orth(h, j, vj, zj, w, mode);
          CK(cudaStreamEndCapture(s, &gr));
          const cudaError_t ie = cudaGraphInstantiate(&gx[j], gr, 0);
          cudaGraphDestroy(gr);
          CK(ie);
          // the capture went through the counting launch wrappers; replays are
          // credited with the same number of kernels
          gc[j] = t_launch_count - l0;
          g_launch_count.fetch_sub(gc[j]);
        }
        CK(cudaGraphLaunch(gx[j], s));
        g_launch_count.fetch_add(gc[j]);
      } else {
        arnoldi_orth(h, j, vj, zj, w, mode);
      }
      CK(cudaMemcpyAsync(h->hflag, h->flag, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h->prof_used) prof_flush(h);
      ++iters;
      reorths += h->hflag[4] != 0.0 ? 1 : 0;
      k = j + 1;
      if (h->hflag[2] != 0.0) { numeric = true; break; }
      if (h->hflag[0] <= tol || h->hflag[3] != 0.0 || iters >= h->opt.max_iters) break;
    }
    if (numeric) { status = SD_E_NUMERIC; break; }
    launch_backsolve(h->st, k, m, sc + sd_handle::S_Y, nullptr, s);
    launch_axpy_multi(x + o, h->Z + o, vs, sc + sd_handle::S_Y, k, len, nullptr, s);
  }
  CK(cudaGetLastError());
  if (info) {
    info->iters = iters;
    info->restarts = restarts;
    info->relres = relres;
    info->status = status;
    info->reorths = reorths;
    // the last residual b - A x is still in V_0 unless a cycle ended on NaN/Inf
    info->relres_v = info->relres_pff = info->relres_pm = -1.0;
    if (mode == MODE_MONO && status != SD_E_NUMERIC) CKR(queue_block_residuals(h, bnorm));
  }
  return status;
}

// Order of the two subdomain solves: the porous medium first unless Sec. 3's
// order (free flow first, velocity prescribed; traction sides only) is asked
// for.
bool partitioned_ff_first(const sd_options& o) { return o.coupling_order == SD_ORDER_FF_FIRST; }

// Partitioned coupling of Sec. 3 for one time step (include/sd.h,
// SD_PARTITIONED): the Darcy solve with the interface flux given, the
// free-flow solve with the pressure below the interface given, and the
// IQN-ILS update of the interface velocity, until the exchanged pressure and
// velocity both settle.  Both subdomain iterates live in the state vector x
// (disjoint ranges), so the converged x is the coupled state.
int step_partitioned(sd_handle* h, sd_step_info* info) {
  cudaStream_t s = h->s;
  const Geom& g = h->g;
  IqnState& q = h->iqn;
  const int n = h->n;
  const Coef<double> c = coef64(h, 0);
  double* vG = h->x + g.ov;                                       // interface faces of the state
  const double* pTop = h->x + g.opm + (long long)(n - 1) * g.P;  // pm cells below the interface
  const bool ff_first = partitioned_ff_first(h->opt);
  CK(cudaMemcpyAsync(q.v, vG, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemsetAsync(q.scal, 0, sizeof(double) * 8, s));
  int iters = 0, it = 0, status = SD_OK, reorths = 0;
  bool conv = false;
  const double eps2 = h->opt.coupling_eps * h->opt.coupling_eps;
  while (it < h->opt.coupling_max) {
    ++it;
    sd_step_info sp, sf;
    std::memset(&sp, 0, sizeof(sp));
    std::memset(&sf, 0, sizeof(sf));
    int rc;
    if (ff_first) {
      // free flow with the interface velocity prescribed, then the Darcy rows with
      // the interface pressure it returns
      launch_dn_iface(3, c, nullptr, h->b, q.v, h->bsub, s);
      CK(cudaMemcpyAsync(vG, q.v, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      rc = fgmres(h, h->bsub, h->x, &sf, MODE_FFD);
      iters += sf.iters;
      reorths += sf.reorths;
      if (rc == SD_E_CUDA || rc == SD_E_NOMEM) return rc;
      if (rc != SD_OK) { status = rc; break; }
      launch_apply_ff(c, h->x, nullptr, h->V, 0, s);
      launch_dn_iface(0, c, h->V, h->b, h->x, q.pG, s);
      launch_dn_iface(2, c, nullptr, h->b, q.pG, h->bsub, s);
      rc = fgmres(h, h->bsub, h->x, &sp, MODE_PMD);
      iters += sp.iters;
      reorths += sp.reorths;
      if (rc == SD_E_CUDA || rc == SD_E_NOMEM) return rc;
      if (rc != SD_OK) { status = rc; break; }
      launch_dn_iface(1, c, h->x, nullptr, q.pG, q.vt, s);
      launch_iqn(q, q.vt, q.pG, s);
    } else {
      launch_dn_rhs_pm(g, h->b, q.v, h->bsub, s);
      rc = fgmres(h, h->bsub, h->x, &sp, MODE_PM);
      iters += sp.iters;
      reorths += sp.reorths;
      if (rc == SD_E_CUDA || rc == SD_E_NOMEM) return rc;
      if (rc != SD_OK) { status = rc; break; }
      launch_dn_rhs_ff(g, h->b, pTop, h->bsub, s);
      rc = fgmres(h, h->bsub, h->x, &sf, MODE_FF);
      iters += sf.iters;
      reorths += sf.reorths;
      if (rc == SD_E_CUDA || rc == SD_E_NOMEM) return rc;
      if (rc != SD_OK) { status = rc; break; }
      launch_iqn(q, vG, pTop, s);
    }
    CK(cudaMemcpyAsync(h->hflag + 8, q.scal + 2, 4 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double* f = h->hflag + 8;  // |dp|^2 (negative: first evaluation), |p|^2, |dv|^2, |v~|^2
    if (!std::isfinite(f[0]) || !std::isfinite(f[1]) || !std::isfinite(f[2]) || !std::isfinite(f[3])) {
      status = SD_E_NUMERIC;
      break;
    }
    if (f[0] >= 0.0 && f[0] <= eps2 * f[1] && f[2] <= eps2 * f[3]) {
      conv = true;
      break;
    }
    // neither subdomain solve moved its state: the interface data changed by
    // less than the solves resolve, and no further evaluation can change x
    if (it > 1 && sp.iters == 0 && sf.iters == 0) {
      conv = true;
      break;
    }
  }
  if (status == SD_OK && !conv) status = SD_E_NOCONV;
  // residual of the coupled state in the monolithic system
  double* sc = h->scal;
  apply_op(h, MODE_MONO, h->x, h->b, h->V);
  launch_dot(h->V, h->V, g.len, h->partial, h->nblk, sc + sd_handle::S_B2, s);
  launch_dot(h->b, h->b, g.len, h->partial, h->nblk, sc + sd_handle::S_BN, s);
  CK(cudaMemcpyAsync(h->hflag + 10, sc + sd_handle::S_B2, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(h->hflag + 11, sc + sd_handle::S_BN, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (info) {
    const double r2 = h->hflag[10], b2 = h->hflag[11];
    info->iters = iters;
    info->restarts = 0;
    info->relres = b2 > 0 ? std::sqrt(r2 / b2) : std::sqrt(r2);
    info->status = status;
    info->reorths = reorths;
    info->coupling_iters = it;
    CKR(block_residuals(h, std::sqrt(b2), info));
  }
  return status;
}

// Time function of the boundary and source data B1: 1 + t for the
// manufactured cases; for the pressure-driven problem (Sec. 5) the inflow
// pressure, a half cosine from 0 to bc_dp over [0, t_end] (t_end = bc_tend,
// or 25 steps when 0), constant afterwards.
double data_scale(const sd_handle* h, double t) {
  if (h->opt.bc != SD_BC_PAPER) return 1.0 + t;
  const double te = h->opt.bc_tend > 0 ? h->opt.bc_tend : 25.0 * h->dt;
  const double s = t < te ? t : te;
  return h->opt.bc_dp * 0.5 * (1.0 - std::cos(3.14159265358979323846 * s / te));
}

// Right-hand side and initial guess of the next implicit-Euler step, queued on s.
int step_rhs(sd_handle* h, cudaStream_t s) {
  const double cm = h->g.h * h->g.h / h->dt;
  const double tn = h->t + h->dt;
  const int lat = h->opt.bc != SD_BC_MMS;
  const bool extra = h->opt.extrapolate && h->have_prev;
  const int order = extra ? std::max(0, std::min(h->opt.extrapolate, h->levels - 1)) : 0;
  if (h->ydepth) {
    // the first residual is formed from the operator history when it reaches
    // back as far as the extrapolation; the history shifts either way
    if (h->ylev > 0)
      launch_yhist(h->Y, h->ydepth, h->V, h->g.len, order, h->ylev >= order + 1 ? 1 : 0, h->scal + sd_handle::S_RH,
                   s);
    else
      CK(cudaMemsetAsync(h->scal + sd_handle::S_RH, 0, sizeof(double), s));
  }
  if (extra) {
    // extrapolate over the solved levels only, up to the option's order; the
    // history shifts, and x_m then holds x^n, the mass-term source
    launch_extrapolate(h->x, h->xm, h->xmm, h->x3, h->g.len, order, s);
    launch_rhs(h->g, lat, cm, h->B0, h->B1, data_scale(h, tn), h->xm, h->b, h->x, s);
  } else {
    // the previous state is both the mass-term source and the initial guess
    CK(cudaMemcpyAsync(h->xm, h->x, sizeof(double) * h->g.len, cudaMemcpyDeviceToDevice, s));
    launch_rhs(h->g, lat, cm, h->B0, h->B1, data_scale(h, tn), h->x, h->b, h->x, s);
  }
  h->have_prev = true;
  h->levels = std::min(h->levels + 1, 4);  // the step's solve adds a solved level
  return SD_OK;
}

int copy_in_dense(sd_handle* h, const double* src, long long count) {
  CK(cudaMemcpyAsync(h->stage, src, sizeof(double) * count,
                     is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->s));
  return SD_OK;
}

int copy_out(sd_handle* h, double* dst, const double* src, long long count) {
  CK(cudaMemcpyAsync(dst, src, sizeof(double) * count,
                     is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->s));
  return SD_OK;
}

int validate(const sd_grid* grid, double mu, double alpha, double dt, const sd_options* o) {
  if (!grid || grid->nx != grid->ny || grid->nx < 2) return SD_E_INVAL;
  if (!(mu > 0) || !(alpha > 0) || !(dt > 0) || !std::isfinite(mu) || !std::isfinite(alpha) || !std::isfinite(dt))
    return SD_E_INVAL;
  if (o->restart < 1 || o->restart > 30 || !(o->rtol > 0) || o->max_iters < 1) return SD_E_INVAL;
  if (o->precision != SD_FP64 && o->precision != SD_MIXED) return SD_E_INVAL;
  if (o->precond < SD_TRI_SCHUR || o->precond > SD_PV_BGS_I) return SD_E_INVAL;
  if (o->bc != SD_BC_MMS && o->bc != SD_BC_MMS_TRACTION && o->bc != SD_BC_PAPER) return SD_E_INVAL;
  if (!std::isfinite(o->bc_dp) || !(o->bc_tend >= 0) || !std::isfinite(o->bc_tend)) return SD_E_INVAL;
  if (o->cheb_degree < 1 || o->cheb_degree > 8 || o->coarsest < 2 || !(o->schur_gamma > 0) || !(o->cheb_ratio > 1))
    return SD_E_INVAL;
  if (o->orth < 0 || o->orth > 1 || !(o->reorth_eta > 0) || o->reorth_eta > 1) return SD_E_INVAL;
  if (o->graph < 0 || o->graph > 2) return SD_E_INVAL;
  if (o->extrapolate < 0 || o->extrapolate > 3) return SD_E_INVAL;
  if (o->darcy_coupled < 0 || o->darcy_coupled > 2) return SD_E_INVAL;
  if (o->tile < 0 || o->tile > 2) return SD_E_INVAL;
  if (o->tile_rows != 0 && o->tile_rows != 4 && o->tile_rows != 8 && o->tile_rows != 16) return SD_E_INVAL;
  if (o->coupling != SD_MONOLITHIC && o->coupling != SD_PARTITIONED) return SD_E_INVAL;
  if (o->coupling_order < SD_ORDER_AUTO || o->coupling_order > SD_ORDER_FF_FIRST) return SD_E_INVAL;
  // the free flow with a prescribed interface velocity is singular on Dirichlet sides
  if (o->coupling == SD_PARTITIONED && o->coupling_order == SD_ORDER_FF_FIRST && o->bc == SD_BC_MMS)
    return SD_E_INVAL;
  if (o->coupling == SD_PARTITIONED &&
      (o->coupling_max < 1 || o->coupling_columns < 1 || o->coupling_columns > 30 || !(o->coupling_eps > 0) ||
       !(o->coupling_omega > 0) || !(o->coupling_omega <= 2) || !(o->coupling_rtol >= 0) ||
       !(o->coupling_rtol < 1)))
    return SD_E_INVAL;
  if (o->cheb_degree_coarse < 0 || o->cheb_degree_coarse > 8 || o->schur_degree < 0 || o->schur_degree > 8)
    return SD_E_INVAL;
  if (o->geometry != SD_GEO_SQUARE && o->geometry != SD_GEO_CHANNEL) return SD_E_INVAL;
  if (o->darcy_schur < 0 || o->darcy_schur > 1) return SD_E_INVAL;
  // the channel runs the monolithic coupling only
  if (o->geometry == SD_GEO_CHANNEL && o->coupling != SD_MONOLITHIC) return SD_E_INVAL;
  int n = grid->nx, L = level_count(n, coarsest_of(*o));
  for (int l = 1; l < L; ++l) n /= 2;
  if (n > 16) return SD_E_INVAL;  // coarsest grid must stay small for the dense solve
  if (o->geometry == SD_GEO_CHANNEL && n > CHANNEL_COARSEST_MAX) return SD_E_INVAL;
  return SD_OK;
}

void init_layout(sd_handle* h) {
  const int geo = h->opt.geometry == SD_GEO_CHANNEL ? 1 : 0;
  h->g = make_geom(h->n, geo);
  h->nlev = level_count(h->n, coarsest_of(h->opt));
  h->geo.clear();
  int nl = h->n;
  for (int l = 0; l < h->nlev; ++l) {
    h->geo.push_back(make_geom(nl, geo));
    nl /= 2;
  }
  h->m = h->opt.restart;
  h->lenA = (h->g.len + 31) / 32 * 32;
  h->nblk = reduce_blocks(h->g.len);
}

int create_impl(const sd_grid* grid, double mu, const double* K, double alpha, double dt, const sd_options* opt,
                sd_handle** out) {
  sd_options o;
  sd_options_default(&o);
  if (opt) o = *opt;
  if (!out || !K) return SD_E_INVAL;
  CKR(validate(grid, mu, alpha, dt, &o));
  const int n = grid->nx;
  // K must be positive and finite (checked on the host copy)
  std::vector<double> Kh((size_t)n * n);
  if (is_device_ptr(K)) CK(cudaMemcpy(Kh.data(), K, sizeof(double) * n * n, cudaMemcpyDeviceToHost));
  else std::memcpy(Kh.data(), K, sizeof(double) * n * n);
  for (double kv : Kh)
    if (!(kv > 0) || !std::isfinite(kv)) return SD_E_INVAL;
  sd_handle* h = new (std::nothrow) sd_handle();
  if (!h) return SD_E_NOMEM;
  h->n = n; h->mu = mu; h->alpha = alpha; h->dt = dt; h->opt = o;
  init_layout(h);
  // the setup's launches use programmatic dependent launch as the steps do
  struct PdlScope {
    int prev;
    explicit PdlScope(int on) : prev(t_pdl) { t_pdl = on; }
    ~PdlScope() { t_pdl = prev; }
  } pdl_scope(o.pdl);
  auto fail = [&](int code) { sd_destroy(h); return code; };
  if (o.stream) {
    h->s = (cudaStream_t)o.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->s, cudaStreamNonBlocking) != cudaSuccess) return fail(SD_E_CUDA);
    h->own_stream = true;
  }
  h->ar = Arena();
  h->ar.plan = true;
  plan_all(h);
  const size_t bytes = h->ar.off;
  h->ar.plan = false;
  h->ar.off = 0;
  if (cudaMalloc(&h->ar.base, bytes) != cudaSuccess) { cudaGetLastError(); h->ar.base = nullptr; return fail(SD_E_NOMEM); }
  if (cudaMemsetAsync(h->ar.base, 0, bytes, h->s) != cudaSuccess) return fail(SD_E_CUDA);
  plan_all(h);
  if (cudaHostAlloc(&h->hflag, 32 * sizeof(double), cudaHostAllocDefault) != cudaSuccess) return fail(SD_E_CUDA);
  if (cudaStreamCreateWithFlags(&h->s2, cudaStreamNonBlocking) != cudaSuccess) return fail(SD_E_CUDA);
  if (cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(SD_E_CUDA);
  for (int q = 0; q < 5; ++q) {
    h->gexec[q].assign(h->m, nullptr);
    h->gcount[q].assign(h->m, 0);
  }
  if (prepare_coarse_cycle<float>() != 0 || prepare_coarse_cycle<double>() != 0) return fail(SD_E_CUDA);
  if (cudaEventCreate(&h->e0) != cudaSuccess || cudaEventCreate(&h->e1) != cudaSuccess) return fail(SD_E_CUDA);
  cudaStream_t s = h->s;
  // permeability hierarchy (geometric means of 2 x 2 children)
  if (cudaMemcpyAsync(h->stage, Kh.data(), sizeof(double) * n * n, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return fail(SD_E_CUDA);
  launch_pack_K(h->stage, n, h->Klev[0], h->geo[0].P, s);
  for (int l = 1; l < h->nlev; ++l)
    launch_coarsen_K(h->Klev[l - 1], h->geo[l - 1].n, h->geo[l - 1].P, h->Klev[l], h->geo[l].P, s);
  const int lat = o.bc != SD_BC_MMS;
  for (int l = 0; l < h->nlev; ++l) {
    LevelCoef<double>& C = h->c64[l];
    const Geom& g = h->geo[l];
    launch_setup_coef<double>(h->Klev[l], g.n, g.n, g.P, mu, alpha, lat, 0, 0, g.n, g.nx, g.iw, C.w, C.rg, C.Tx,
                              C.Ty, s);
    // the preconditioner's Darcy block: Ty, with the interface's Schur
    // correction on the top faces in the monolithic solve
    if (cudaMemcpyAsync(C.TyR, C.Ty, sizeof(double) * (g.n + 1) * g.P, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(SD_E_CUDA);
    if (o.darcy_schur && o.coupling == SD_MONOLITHIC)
      launch_darcy_schur_top(C.TyR, C.w, C.rg, g.n, g.nx, g.iw, g.P, mu, g.h * g.h / dt, g.h, lat, s);
  }
  // pressure Laplacian B^T B / h^2 over the free-flow cells: TPFA with K / mu
  // = 1 (the Krylov slots hold the unit permeability, free during setup); its
  // bottom faces are Dirichlet below the interface (the half control volume
  // of v_Gamma), no-flow beside it
  for (int l = 0; l < h->nlev; ++l) {
    LevelCoef<double>& C = h->c64[l];
    const Geom& g = h->geo[l];
    launch_fill_K(h->V, g.nx, g.n, g.P, mu, s);
    launch_setup_coef<double>(h->V, g.n, g.nx, g.P, mu, alpha, lat, lat, g.iw, g.iw + g.n, g.nx, g.iw, C.wP, C.rgP,
                              C.TxP, C.TyP, s);
  }
  const Coef<double> c0 = coef64(h, 0);
  launch_mms_terms(c0, o.bc, h->Klev[0], h->B0, h->B1, s);
  if (o.bc == SD_BC_PAPER) {  // the pressure-driven problem starts from rest
    if (cudaMemsetAsync(h->x, 0, sizeof(double) * h->g.len, s) != cudaSuccess) return fail(SD_E_CUDA);
  } else {
    launch_mms_exact(h->g, mu, 0.0, h->x, s);
  }
  int rc = (h->opt.precision == SD_MIXED) ? setup_mg<float>(h, h->mg32) : setup_mg<double>(h, h->mg64);
  if (rc != SD_OK) return fail(rc);
  // the setup used the Krylov bases as scratch: clear them (padding must be zero)
  if (cudaMemsetAsync(h->V, 0, sizeof(double) * (h->m + 1) * h->lenA, s) != cudaSuccess ||
      cudaMemsetAsync(h->Z, 0, sizeof(double) * h->m * h->lenA, s) != cudaSuccess)
    return fail(SD_E_CUDA);
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) return fail(SD_E_CUDA);
  h->t = 0.0;
  h->step = 0;
  *out = h;
  return SD_OK;
}

}  // namespace

// ====================================================== lockstep batches
// Instances with the same grid, viscosity, time step and options have
// buffers at the same offsets inside their allocations, so one launch can
// serve all of them (Bat in sd_internal.cuh): blockIdx.z picks the instance
// and every pointer of instance 0 is moved by that instance's offset.  The
// FGMRES iterations run in lockstep: each Arnoldi step is one captured graph
// for the whole batch, and an instance that has met its own stopping test
// is made idle (its blocks return at once) while the others go on.  Every
// instance does exactly the arithmetic of its single-instance solve (same
// per-instance reductions, same coefficients), so its result is bitwise the
// same.
namespace sdk {

int handle_grid(const sd_handle* h) { return h->n; }
long long handle_dof(const sd_handle* h) { return dof_of(h); }

bool can_lockstep(const sd_handle* a, const sd_handle* b) {
  const sd_options& x = a->opt;
  const sd_options& y = b->opt;
  const bool same_opt = x.restart == y.restart && x.rtol == y.rtol && x.max_iters == y.max_iters &&
                        x.precision == y.precision && x.precond == y.precond && x.bc == y.bc &&
                        x.cheb_degree == y.cheb_degree && x.cheb_degree_coarse == y.cheb_degree_coarse &&
                        x.schur_degree == y.schur_degree && x.coarsest == y.coarsest &&
                        x.schur_gamma == y.schur_gamma && x.cheb_ratio == y.cheb_ratio &&
                        x.schur_mass == y.schur_mass && x.fuse_coarse == y.fuse_coarse && x.orth == y.orth &&
                        x.reorth_eta == y.reorth_eta && x.extrapolate == y.extrapolate && x.graph == y.graph &&
                        x.pdl == y.pdl && x.tile == y.tile && x.tile_rows == y.tile_rows &&
                        x.darcy_coupled == y.darcy_coupled && x.bc_dp == y.bc_dp && x.bc_tend == y.bc_tend &&
                        x.geometry == y.geometry && x.darcy_schur == y.darcy_schur &&
                        x.coupling == SD_MONOLITHIC &&
                        y.coupling == SD_MONOLITHIC;
  return same_opt && a->n == b->n && a->mu == b->mu && a->dt == b->dt && a->ar.off == b->ar.off &&
         a->nlev == b->nlev && a->prof_id < 0 && b->prof_id < 0;
}

namespace {

struct Lockstep {
  std::vector<sd_handle*> hs;
  int B = 0;
  long long* off_dev = nullptr;
  int* act_dev = nullptr;
  double* gat_dev = nullptr;
  double* gat_host = nullptr;  // pinned
  std::vector<int> act;
  std::vector<cudaGraphExec_t> gexec;
  std::vector<long long> gcount;
  ~Lockstep() {
    for (auto& g : gexec)
      if (g) cudaGraphExecDestroy(g);
    if (off_dev) cudaFree(off_dev);
    if (act_dev) cudaFree(act_dev);
    if (gat_dev) cudaFree(gat_dev);
    if (gat_host) cudaFreeHost(gat_host);
  }
};

// makes the calling thread's launches serve the whole batch
struct BatScope {
  Bat saved;
  int saved_n;
  BatScope(const Lockstep& L) : saved(t_bat), saved_n(t_bat_n) {
    t_bat.off = L.off_dev;
    t_bat.act = L.act_dev;
    t_bat_n = L.B;
  }
  ~BatScope() {
    t_bat = saved;
    t_bat_n = saved_n;
  }
};

// upload the idle mask (from pageable memory: the copy has taken the data
// when the call returns)
int set_act(Lockstep& L, cudaStream_t s) {
  CK(cudaMemcpyAsync(L.act_dev, L.act.data(), sizeof(int) * L.B, cudaMemcpyHostToDevice, s));
  return SD_OK;
}

// every instance's src[0..count) into L.gat_host[z * count + t]
int gather(Lockstep& L, const double* src, int count, cudaStream_t s) {
  launch_gather_inst(src, count, L.gat_dev, s);
  CK(cudaMemcpyAsync(L.gat_host, L.gat_dev, sizeof(double) * count * L.B, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return SD_OK;
}

int fgmres_lockstep(Lockstep& L, std::vector<sd_step_info>& si) {
  sd_handle* h = L.hs[0];
  cudaStream_t s = h->s;
  const int B = L.B;
  const long long len = h->g.len, vs = h->lenA;
  const int m = h->m, nb = h->nblk;
  const Coef<double> c = coef64(h, 0);
  double* sc = h->scal;
  BatScope bs(L);
  std::vector<int> iters(B, 0), restarts(B, 0), reorths(B, 0), status(B, SD_OK);
  std::vector<double> relres(B, 0.0), bnorm(B), tol(B);
  std::vector<char> live(B, 1), cyc(B, 0), numeric(B, 0);
  L.act.assign(B, 1);
  CKR(set_act(L, s));
  // ||b|| and the first true residual, gathered together (S_B2, S_BN adjacent)
  resid_norms(h, MODE_MONO, h->x, h->b, true);  // V_0 = b - A x
  CKR(gather(L, sc + sd_handle::S_B2, 2, s));
  for (int i = 0; i < B; ++i) {
    bnorm[i] = std::sqrt(L.gat_host[(size_t)i * 2 + 1]);
    tol[i] = h->opt.rtol * (bnorm[i] > 0 ? bnorm[i] : 1.0);
    L.gat_host[i] = L.gat_host[(size_t)i * 2];  // beta^2 where the loop reads it
  }
  bool first = true;
  for (;;) {
    if (!first) {
      for (int i = 0; i < B; ++i) L.act[i] = live[i];
      CKR(set_act(L, s));
      resid_norms(h, MODE_MONO, h->x, h->b, false);  // V_0 = b - A x
      CKR(gather(L, sc + sd_handle::S_B2, 1, s));
    }
    first = false;
    bool any = false;
    for (int i = 0; i < B; ++i) {
      cyc[i] = 0;
      if (!live[i]) continue;
      const double beta = std::sqrt(L.gat_host[i]);
      relres[i] = bnorm[i] > 0 ? beta / bnorm[i] : beta;
      if (!std::isfinite(beta)) { status[i] = SD_E_NUMERIC; live[i] = 0; continue; }
      if (beta <= tol[i]) { live[i] = 0; continue; }
      if (iters[i] >= h->opt.max_iters) { status[i] = SD_E_NOCONV; live[i] = 0; continue; }
      cyc[i] = 1;
      restarts[i] += 1;
      any = true;
    }
    if (!any) break;
    for (int i = 0; i < B; ++i) L.act[i] = cyc[i];
    CKR(set_act(L, s));
    launch_init_cycle(h->st, m, sc + sd_handle::S_B2, h->flag, s, sc + sd_handle::S_VSC);
    for (int j = 0; j < m; ++j) {
      double* vj = h->V + (long long)j * vs;
      double* zj = h->Z + (long long)j * vs;
      double* w = h->V + (long long)(j + 1) * vs;
      if (h->opt.graph) {
        if (!L.gexec[j]) {
          cudaGraph_t gr = nullptr;
          const long long l0 = t_launch_count;
          CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
          arnoldi_orth(h, j, vj, zj, w);
          CK(cudaStreamEndCapture(s, &gr));
          const cudaError_t ie = cudaGraphInstantiate(&L.gexec[j], gr, 0);
          cudaGraphDestroy(gr);
          CK(ie);
          L.gcount[j] = t_launch_count - l0;
          g_launch_count.fetch_sub(L.gcount[j]);
        }
        CK(cudaGraphLaunch(L.gexec[j], s));
        g_launch_count.fetch_add(L.gcount[j]);
      } else {
        arnoldi_orth(h, j, vj, zj, w);
      }
      CKR(gather(L, h->flag, 6, s));
      bool running = false;
      for (int i = 0; i < B; ++i) {
        if (!L.act[i]) continue;
        const double* f = L.gat_host + (size_t)i * 6;
        iters[i] += 1;
        reorths[i] += f[4] != 0.0 ? 1 : 0;
        if (f[2] != 0.0) {
          numeric[i] = 1;
          L.act[i] = 0;
        } else if (f[0] <= tol[i] || f[3] != 0.0 || iters[i] >= h->opt.max_iters) {
          L.act[i] = 0;
        } else {
          running = true;
        }
      }
      if (!running) break;
      CKR(set_act(L, s));
    }
    // solution update of every instance that took part in the cycle, each
    // with its own number of basis vectors (flag[5], written by k_givens)
    for (int i = 0; i < B; ++i) {
      if (numeric[i]) {
        status[i] = SD_E_NUMERIC;
        live[i] = 0;
        cyc[i] = 0;
      }
      L.act[i] = cyc[i];
    }
    CKR(set_act(L, s));
    launch_backsolve(h->st, m, m, sc + sd_handle::S_Y, h->flag + 5, s);
    launch_axpy_multi(h->x, h->Z, vs, sc + sd_handle::S_Y, m, len, h->flag + 5, s);
  }
  // per-block residual norms: every instance's last residual left them in
  // its S_BLK (its kernels were idle since), unless a cycle of it ended on
  // NaN/Inf
  L.act.assign(B, 1);
  CKR(set_act(L, s));
  CKR(gather(L, sc + sd_handle::S_BLK, 3, s));
  CK(cudaGetLastError());
  for (int i = 0; i < B; ++i) {
    si[i].iters = iters[i];
    si[i].restarts = restarts[i];
    si[i].relres = relres[i];
    si[i].status = status[i];
    si[i].reorths = reorths[i];
    const double d = bnorm[i] > 0 ? bnorm[i] : 1.0;
    const bool ok = status[i] != SD_E_NUMERIC;
    si[i].relres_v = ok ? std::sqrt(L.gat_host[(size_t)i * 3]) / d : -1.0;
    si[i].relres_pff = ok ? std::sqrt(L.gat_host[(size_t)i * 3 + 1]) / d : -1.0;
    si[i].relres_pm = ok ? std::sqrt(L.gat_host[(size_t)i * 3 + 2]) / d : -1.0;
  }
  return SD_OK;
}

// ------------------------------------- lockstep groups as one graph
// The launches of the calling host thread serve no batch (the group control
// kernels are single CTAs over all instances, the right-hand sides are
// single-instance launches).
struct NoBatScope {
  Bat saved;
  int saved_n;
  NoBatScope() : saved(t_bat), saved_n(t_bat_n) {
    t_bat.off = nullptr;
    t_bat.act = nullptr;
    t_bat_n = 1;
  }
  ~NoBatScope() {
    t_bat = saved;
    t_bat_n = saved_n;
  }
};

// One lockstep group's whole FGMRES solve as a branch of graph `top`: the
// steps of fgmres_lockstep with its host decisions taken by the k_grp_*
// kernels (the same values, the same order), a WHILE node over restart
// cycles and IF nodes over the Arnoldi steps of a cycle.  pre: the kernels
// outside the loops (those inside are counted on the device, instance 0's
// C_KERN).
int build_group_branch(Lockstep& L, cudaGraph_t top, long long* pre) {
  sd_handle* h = L.hs[0];
  cudaStream_t s = h->s;
  const long long len = h->g.len, vs = h->lenA;
  const int m = h->m, maxit = h->opt.max_iters;
  double* sc = h->scal;
  double* ctl = sc + sd_handle::S_CTL;
  const int saved_pdl = t_pdl, pdl = h->opt.pdl;
  t_pdl = pdl;
  const long long l_start = t_launch_count;
  BatScope bs(L);
  std::vector<cudaGraphNode_t> deps;
  bool capturing = false;
  cudaError_t err = cudaSuccess;
  auto begin = [&](cudaGraph_t g, bool after) {
    if (err != cudaSuccess) return false;
    err = cudaStreamBeginCaptureToGraph(s, g, after ? deps.data() : nullptr, nullptr, after ? deps.size() : 0,
                                        cudaStreamCaptureModeThreadLocal);
    capturing = err == cudaSuccess;
    return capturing;
  };
  auto end = [&](bool keep) {
    if (!capturing) return;
    if (keep && err == cudaSuccess) {
      cudaStreamCaptureStatus st;
      const cudaGraphNode_t* d = nullptr;
      size_t nd = 0;
      err = cudaStreamGetCaptureInfo(s, &st, nullptr, nullptr, &d, nullptr, &nd);
      if (err == cudaSuccess) deps.assign(d, d + nd);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(s, &g);
    capturing = false;
    if (err == cudaSuccess) err = e2;
    if (err == cudaSuccess) err = cudaGetLastError();
  };
  auto cond = [&](cudaGraph_t g, cudaGraphConditionalHandle hd, cudaGraphConditionalNodeType type,
                  cudaGraph_t* body) {
    if (err != cudaSuccess) return;
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hd;
    np.conditional.type = type;
    np.conditional.size = 1;
    cudaGraphNode_t nd = nullptr;
    err = cudaGraphAddNode(&nd, g, deps.data(), nullptr, deps.size(), &np);
    if (err != cudaSuccess) return;
    *body = np.conditional.phGraph_out[0];
    deps.assign(1, nd);
  };
  auto step = [&](int j) {
    const long long l0 = t_launch_count;
    double* vj = h->V + (long long)j * vs;
    double* zj = h->Z + (long long)j * vs;
    double* w = h->V + (long long)(j + 1) * vs;
    arnoldi_orth(h, j, vj, zj, w);
    return t_launch_count - l0;
  };
  cudaGraphConditionalHandle loop = 0;
  CondSet cs = {};
  cs.n = m;
  err = cudaGraphConditionalHandleCreate(&loop, top, 0, cudaGraphCondAssignDefault);
  for (int j = 1; j < m && err == cudaSuccess; ++j)
    err = cudaGraphConditionalHandleCreate(&cs.c[j], top, 0, cudaGraphCondAssignDefault);
  // every instance active, ||b|| and the first true residual, the first decisions
  if (begin(top, false)) {
    const long long l0 = t_launch_count;
    {
      NoBatScope nb;
      launch_grp_act_all(L.act_dev, L.B, s);
    }
    resid_norms(h, MODE_MONO, h->x, h->b, true);
    {
      NoBatScope nb;
      launch_grp_begin(L.off_dev, L.B, sc + sd_handle::S_BN, ctl, h->opt.rtol, s);
      launch_grp_restart(L.off_dev, L.act_dev, L.B, sc + sd_handle::S_B2, ctl, maxit, maxit + 2, 0.0, loop, s);
    }
    *pre = t_launch_count - l0;
    end(true);
  }
  cudaGraph_t wbody = nullptr;
  cond(top, loop, cudaGraphCondTypeWhile, &wbody);
  deps.clear();
  if (begin(wbody, false)) {
    const long long l0 = t_launch_count;
    {
      NoBatScope nb;
      launch_cycle_head(cs, s);
    }
    launch_init_cycle(h->st, m, sc + sd_handle::S_B2, h->flag, s, sc + sd_handle::S_VSC);
    step(0);
    const long long k = t_launch_count - l0 + 1;
    {
      NoBatScope nb;
      launch_grp_step(L.off_dev, L.act_dev, L.B, h->flag, ctl, maxit, (double)k, m > 1, m > 1 ? cs.c[1] : 0, s);
    }
    end(true);
  }
  for (int j = 1; j < m; ++j) {
    cudaGraph_t ib = nullptr;
    cond(wbody, cs.c[j], cudaGraphCondTypeIf, &ib);
    const std::vector<cudaGraphNode_t> keep = deps;
    if (begin(ib, false)) {
      const long long k = step(j) + 1;
      NoBatScope nb;
      launch_grp_step(L.off_dev, L.act_dev, L.B, h->flag, ctl, maxit, (double)k, j + 1 < m,
                      j + 1 < m ? cs.c[j + 1] : 0, s);
      end(false);
    }
    deps = keep;
  }
  // the update of x of the instances that took part (each with its own k,
  // flag[5]), then every live instance's true residual and the next
  // decisions; no programmatic edge out of a conditional node
  if (begin(wbody, true)) {
    const long long l0 = t_launch_count;
    t_pdl = 0;
    {
      NoBatScope nb;
      launch_grp_cycle_end(L.off_dev, L.act_dev, L.B, ctl, 0.0, s);
    }
    t_pdl = pdl;
    launch_backsolve(h->st, m, m, sc + sd_handle::S_Y, h->flag + 5, s);
    launch_axpy_multi(h->x, h->Z, vs, sc + sd_handle::S_Y, m, len, h->flag + 5, s);
    {
      NoBatScope nb;
      launch_grp_live(L.off_dev, L.act_dev, L.B, ctl, s);
    }
    resid_norms(h, MODE_MONO, h->x, h->b, false);
    const long long k = t_launch_count - l0 + 1;
    NoBatScope nb;
    launch_grp_restart(L.off_dev, L.act_dev, L.B, sc + sd_handle::S_B2, ctl, maxit, maxit + 2, (double)k, loop, s);
    end(false);
  }
  if (capturing) end(false);
  t_pdl = saved_pdl;
  g_launch_count.fetch_sub(t_launch_count - l_start);
  return err == cudaSuccess ? SD_OK : SD_E_CUDA;
}

}  // namespace

int step_lockstep(sd_handle* const* hs, int count, int nsteps, sd_step_info* const* infos) {
  if (count < 1 || nsteps < 0) return SD_E_INVAL;
  for (int i = 1; i < count; ++i)
    if (!can_lockstep(hs[0], hs[i])) return SD_E_INVAL;
  std::vector<sd_handle*> order(hs, hs + count);
  std::sort(order.begin(), order.end());
  if (std::adjacent_find(order.begin(), order.end()) != order.end()) return SD_E_INVAL;  // no handle twice
  std::vector<std::unique_lock<std::mutex>> locks;
  for (sd_handle* h : order) locks.emplace_back(h->mtx);
  Lockstep L;
  L.hs.assign(hs, hs + count);
  L.B = count;
  sd_handle* h0 = hs[0];
  cudaStream_t s = h0->s;
  t_pdl = h0->opt.pdl;
  std::vector<long long> off(count);
  for (int i = 0; i < count; ++i) {
    off[i] = (long long)(reinterpret_cast<uintptr_t>(hs[i]->ar.base) - reinterpret_cast<uintptr_t>(h0->ar.base));
    CK(cudaStreamSynchronize(hs[i]->s));  // nothing of an instance may still run on its own stream
  }
  CK(cudaMalloc(&L.off_dev, sizeof(long long) * count));
  CK(cudaMalloc(&L.act_dev, sizeof(int) * count));
  CK(cudaMalloc(&L.gat_dev, sizeof(double) * 8 * count));
  CK(cudaHostAlloc(&L.gat_host, sizeof(double) * 8 * count, cudaHostAllocDefault));
  CK(cudaMemcpyAsync(L.off_dev, off.data(), sizeof(long long) * count, cudaMemcpyHostToDevice, s));
  L.gexec.assign(h0->m, nullptr);
  L.gcount.assign(h0->m, 0);
  int first = SD_OK;
  std::vector<sd_step_info> si(count);
  t_bat_misuse = 0;
  for (int k = 0; k < nsteps; ++k) {
    CK(cudaEventRecord(h0->e0, s));
    for (int i = 0; i < count; ++i) CKR(step_rhs(hs[i], s));  // single-instance launches on the batch stream
    std::memset(si.data(), 0, sizeof(sd_step_info) * count);
    const int rc = fgmres_lockstep(L, si);
    if (rc != SD_OK) return rc;
    for (int i = 0; i < count; ++i)
      if (hs[i]->ydepth) hs[i]->ylev = std::min(hs[i]->ylev + 1, hs[i]->ydepth);
    if (t_bat_misuse) {
      snprintf(g_errmsg, sizeof(g_errmsg), "a kernel without batch support was launched in a lockstep batch");
      return SD_E_STATE;
    }
    CK(cudaEventRecord(h0->e1, s));
    CK(cudaEventSynchronize(h0->e1));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h0->e0, h0->e1));
    for (int i = 0; i < count; ++i) {
      sd_handle* h = hs[i];
      h->t += h->dt;
      h->step += 1;
      si[i].ms = ms;
      if (infos && infos[i]) infos[i][k] = si[i];
      if (si[i].status != SD_OK && first == SD_OK) first = si[i].status;
    }
  }
  CK(cudaStreamSynchronize(s));
  return first;
}

// The last batch graph: its groups, their group buffers (the graph addresses
// them) and the instantiated graph, reused by the next call with the same
// groups; sd_destroy of any member drops it.  One graph batch runs at a time.
struct BatchGraphCache {
  std::mutex mu;
  std::vector<std::vector<sd_handle*>> groups;
  std::vector<char> on;  // the groups the graph steps
  std::vector<std::unique_ptr<Lockstep>> Ls;
  std::vector<long long> pre;
  cudaGraphExec_t ex = nullptr;
  void clear() {
    if (ex) cudaGraphExecDestroy(ex);
    ex = nullptr;
    Ls.clear();
    groups.clear();
    on.clear();
    pre.clear();
  }
};
BatchGraphCache& batch_cache() {
  static BatchGraphCache* c = new BatchGraphCache();  // never destroyed: no CUDA call at process exit
  return *c;
}

void drop_batch_graph(const sd_handle* h) {
  BatchGraphCache& C = batch_cache();
  std::lock_guard<std::mutex> lk(C.mu);
  for (const auto& g : C.groups)
    if (std::find(g.begin(), g.end(), h) != g.end()) {
      C.clear();
      return;
    }
}

// Every group's solve of a time step in one graph launch (see
// step_graph_batch in sd_internal.cuh).
int step_graph_batch(const std::vector<std::vector<sd_handle*>>& groups, const std::vector<int>& nsteps,
                     const std::vector<std::vector<sd_step_info*>>& infos) {
  const int G = (int)groups.size();
  if (G == 0) return SD_OK;
  std::vector<sd_handle*> order;
  for (const auto& g : groups) {
    if (g.empty()) return SD_E_INVAL;
    for (int i = 1; i < (int)g.size(); ++i)
      if (!can_lockstep(g[0], g[i])) return SD_E_INVAL;
    if (!can_lockstep(g[0], g[0])) return SD_E_INVAL;  // monolithic, no kernel timing
    order.insert(order.end(), g.begin(), g.end());
  }
  std::sort(order.begin(), order.end());
  if (std::adjacent_find(order.begin(), order.end()) != order.end()) return SD_E_INVAL;
  BatchGraphCache& C = batch_cache();
  std::lock_guard<std::mutex> clk(C.mu);
  std::vector<std::unique_lock<std::mutex>> locks;
  for (sd_handle* h : order) locks.emplace_back(h->mtx);
  constexpr int kGat = 16;  // doubles gathered per instance (the control slots)
  for (const auto& g : groups)
    for (sd_handle* h : g) CK(cudaStreamSynchronize(h->s));  // nothing of an instance may still run on its own stream
  if (C.groups != groups) {
    C.clear();
    C.groups = groups;
    C.on.assign(G, 0);
    C.pre.assign(G, 0);
  }
  std::vector<std::unique_ptr<Lockstep>>& Ls = C.Ls;
  for (size_t gi = Ls.size(); gi < groups.size(); ++gi) {
    const auto& g = groups[gi];
    std::unique_ptr<Lockstep> L(new Lockstep());
    L->hs = g;
    L->B = (int)g.size();
    std::vector<long long> off(g.size());
    for (size_t i = 0; i < g.size(); ++i)
      off[i] = (long long)(reinterpret_cast<uintptr_t>(g[i]->ar.base) - reinterpret_cast<uintptr_t>(g[0]->ar.base));
    CK(cudaMalloc(&L->off_dev, sizeof(long long) * L->B));
    CK(cudaMalloc(&L->act_dev, sizeof(int) * L->B));
    CK(cudaMalloc(&L->gat_dev, sizeof(double) * kGat * L->B));
    CK(cudaHostAlloc(&L->gat_host, sizeof(double) * kGat * L->B, cudaHostAllocDefault));
    CK(cudaMemcpy(L->off_dev, off.data(), sizeof(long long) * L->B, cudaMemcpyHostToDevice));
    Ls.push_back(std::move(L));
  }
  cudaStream_t s0 = groups[0][0]->s;
  struct Events {
    std::vector<cudaEvent_t> ev;
    ~Events() {
      for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    }
  } E;
  E.ev.assign(G + 2, nullptr);
  CK(cudaEventCreate(&E.ev[0]));
  CK(cudaEventCreate(&E.ev[1]));
  for (int g = 0; g < G; ++g) CK(cudaEventCreateWithFlags(&E.ev[2 + g], cudaEventDisableTiming));
  std::vector<char>& built = C.on;
  std::vector<long long>& pre = C.pre;
  const int maxsteps = *std::max_element(nsteps.begin(), nsteps.end());
  const int saved_pdl = t_pdl;
  int first = SD_OK;
  t_bat_misuse = 0;
  for (int k = 0; k < maxsteps; ++k) {
    std::vector<char> on(G);
    for (int g = 0; g < G; ++g) on[g] = nsteps[g] > k;
    if (!C.ex || on != built) {  // (re)build for the groups that step now
      if (C.ex) {
        cudaGraphExecDestroy(C.ex);
        C.ex = nullptr;
      }
      cudaGraph_t top = nullptr;
      CK(cudaGraphCreate(&top, 0));
      int rc = SD_OK;
      for (int g = 0; g < G && rc == SD_OK; ++g)
        if (on[g]) rc = build_group_branch(*Ls[g], top, &pre[g]);
      cudaError_t ie = cudaSuccess;
      if (rc == SD_OK) ie = cudaGraphInstantiate(&C.ex, top, 0);
      cudaGraphDestroy(top);
      if (rc != SD_OK || ie != cudaSuccess) {
        C.clear();
        if (rc != SD_OK) return rc;
        CK(ie);
      }
      if (t_bat_misuse) {
        snprintf(g_errmsg, sizeof(g_errmsg), "a kernel without batch support was launched in a lockstep batch");
        return SD_E_STATE;
      }
      built = on;
    }
    // right-hand sides on each group's stream, the solve graph on s0 after all of them
    CK(cudaEventRecord(E.ev[0], s0));
    for (int g = 0; g < G; ++g) {
      if (!on[g]) continue;
      cudaStream_t sg = groups[g][0]->s;
      CK(cudaStreamWaitEvent(sg, E.ev[0], 0));
      NoBatScope nb;
      t_pdl = groups[g][0]->opt.pdl;
      for (sd_handle* h : groups[g]) CKR(step_rhs(h, sg));
      CK(cudaEventRecord(E.ev[2 + g], sg));
      CK(cudaStreamWaitEvent(s0, E.ev[2 + g], 0));
    }
    t_pdl = saved_pdl;
    CK(cudaGraphLaunch(C.ex, s0));
    CK(cudaEventRecord(E.ev[1], s0));
    for (int g = 0; g < G; ++g)
      if (on[g]) CK(cudaStreamWaitEvent(groups[g][0]->s, E.ev[1], 0));
    CK(cudaEventSynchronize(E.ev[1]));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, E.ev[0], E.ev[1]));
    for (int g = 0; g < G; ++g)
      if (on[g])
        for (sd_handle* h : groups[g])
          if (h->ydepth) h->ylev = std::min(h->ylev + 1, h->ydepth);
    for (int g = 0; g < G; ++g) {
      if (!on[g]) continue;
      Lockstep& L = *Ls[g];
      sd_handle* h0 = groups[g][0];
      double* sc = h0->scal;
      BatScope bs(L);
      CKR(gather(L, sc + sd_handle::S_CTL, C_GROUP_END, s0));
      std::vector<double> ctlv(L.gat_host, L.gat_host + (size_t)C_GROUP_END * L.B);
      CKR(gather(L, sc + sd_handle::S_BLK, 3, s0));
      g_launch_count.fetch_add(pre[g] + (long long)ctlv[C_KERN]);  // instance 0's count
      for (int i = 0; i < L.B; ++i) {
        const double* c = ctlv.data() + (size_t)i * C_GROUP_END;
        sd_step_info si;
        std::memset(&si, 0, sizeof(si));
        si.iters = (int)c[C_ITER];
        si.restarts = (int)c[C_REST];
        si.reorths = (int)c[C_REO];
        si.relres = c[C_REL];
        si.status = c[C_STAT] == C_STAT_NUMERIC ? SD_E_NUMERIC : (c[C_STAT] == C_STAT_NOCONV ? SD_E_NOCONV : SD_OK);
        const double d = c[C_BN] > 0 ? c[C_BN] : 1.0;
        const bool ok = si.status != SD_E_NUMERIC;
        si.relres_v = ok ? std::sqrt(L.gat_host[(size_t)i * 3]) / d : -1.0;
        si.relres_pff = ok ? std::sqrt(L.gat_host[(size_t)i * 3 + 1]) / d : -1.0;
        si.relres_pm = ok ? std::sqrt(L.gat_host[(size_t)i * 3 + 2]) / d : -1.0;
        si.ms = ms;
        sd_handle* h = groups[g][i];
        h->t += h->dt;
        h->step += 1;
        if (!infos.empty() && infos[g][i]) infos[g][i][k] = si;
        if (si.status != SD_OK && first == SD_OK) first = si.status;
      }
    }
  }
  CK(cudaStreamSynchronize(s0));
  return first;
}

}  // namespace sdk

// ================================================================ C ABI
extern "C" {

void sd_options_default(sd_options* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->restart = 30;
  o->rtol = 1e-10;
  o->max_iters = 600;
  o->precision = SD_MIXED;
  o->precond = SD_TRI_SCHUR;
  o->bc = SD_BC_MMS;
  o->cheb_degree = 3;
  o->cheb_degree_coarse = 0;
  o->schur_degree = 1;
  o->coarsest = 16;
  o->fuse_coarse = 1;
  o->orth = 1;
  o->reorth_eta = 1e-3;
  o->extrapolate = 2;
  o->graph = 1;
  o->pdl = 1;
  o->tile = 2;
  o->tile_rows = 0;
  o->darcy_coupled = 1;
  o->coupling = SD_MONOLITHIC;
  o->coupling_max = 100;
  o->coupling_columns = 30;
  o->coupling_eps = 1e-9;
  o->coupling_omega = 0.1;
  o->coupling_order = SD_ORDER_AUTO;
  o->coupling_rtol = 0.0;
  o->bc_dp = 1.0;
  o->bc_tend = 0.0;
  o->schur_gamma = 0.5;
  o->cheb_ratio = 8.0;
  o->schur_mass = 1;
  o->stream = nullptr;
  o->geometry = SD_GEO_SQUARE;
  o->darcy_schur = 1;
}

int64_t sd_dof_count(int32_t n) { return 4 * (int64_t)n * n + 2 * (int64_t)n; }

int64_t sd_dof_count_geometry(int32_t n, int32_t geometry) {
  if (geometry == SD_GEO_CHANNEL) return 10 * (int64_t)n * n + 4 * (int64_t)n;
  return geometry == SD_GEO_SQUARE ? sd_dof_count(n) : -1;
}

int64_t sd_memory_estimate(const sd_grid* grid, const sd_options* opt) {
  sd_options o;
  sd_options_default(&o);
  if (opt) o = *opt;
  if (validate(grid, 1.0, 1.0, 1.0, &o) != SD_OK) return -1;
  sd_handle tmp;
  tmp.n = grid->nx;
  tmp.opt = o;
  init_layout(&tmp);
  tmp.ar = Arena();
  plan_all(&tmp);
  return (int64_t)tmp.ar.off;
}

int sd_create(const sd_grid* grid, double mu, const double* K, double alpha_bj, double dt, const sd_options* opt,
              sd_handle** out) {
  if (out) *out = nullptr;
  return create_impl(grid, mu, K, alpha_bj, dt, opt, out);
}

int sd_step(sd_handle* h, int32_t nsteps, sd_step_info* info) {
  if (!h || nsteps < 0) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  t_pdl = h->opt.pdl;
  int first = SD_OK;
  for (int k = 0; k < nsteps; ++k) {
    const double tn = h->t + h->dt;
    CK(cudaEventRecord(h->e0, h->s));
    CKR(step_rhs(h, h->s));
    sd_step_info si;
    std::memset(&si, 0, sizeof(si));
    const int rc = h->opt.coupling == SD_PARTITIONED ? step_partitioned(h, &si) : fgmres(h, h->b, h->x, &si);
    if (rc == SD_E_CUDA || rc == SD_E_NOMEM) return rc;
    if (h->ydepth) h->ylev = std::min(h->ylev + 1, h->ydepth);  // the solve left A x^n in Y[0]
    CK(cudaEventRecord(h->e1, h->s));
    CK(cudaEventSynchronize(h->e1));
    finish_block_residuals(h, &si);
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, h->e0, h->e1));
    si.ms = ms;
    h->t = tn;
    h->step += 1;
    if (info) info[k] = si;
    if (rc != SD_OK && first == SD_OK) first = rc;
  }
  if (h->prof_used) prof_flush(h);
  return first;
}

int sd_get_fields(sd_handle* h, double* u, double* v, double* p_ff, double* p_pm) {
  if (!h) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  const int n = h->n, nx = h->g.nx;
  launch_unpack(h->g, h->x, h->stage, h->s);
  const long long nu = (long long)n * (nx + 1), nv = (long long)nx * (n + 1), npf = (long long)nx * n;
  if (u) CKR(copy_out(h, u, h->stage, nu));
  if (v) CKR(copy_out(h, v, h->stage + nu, nv));
  if (p_ff) CKR(copy_out(h, p_ff, h->stage + nu + nv, npf));
  if (p_pm) CKR(copy_out(h, p_pm, h->stage + nu + nv + npf, (long long)n * n));
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

int sd_get_state(sd_handle* h, double* t, int64_t* step, double* x, double* xprev) {
  if (!h) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  if (t) *t = h->t;
  if (step) *step = h->step;
  if (x) {
    launch_unpack(h->g, h->x, h->stage, h->s);
    CKR(copy_out(h, x, h->stage, dof_of(h)));
  }
  if (xprev) {
    CK(cudaStreamSynchronize(h->s));
    launch_unpack(h->g, h->have_prev ? h->xm : h->x, h->stage, h->s);
    CKR(copy_out(h, xprev, h->stage, dof_of(h)));
  }
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

int sd_set_state(sd_handle* h, double t, int64_t step, const double* x, const double* xprev) {
  if (!h || !x) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  CKR(copy_in_dense(h, x, dof_of(h)));
  launch_pack(h->g, h->stage, h->x, h->s);
  CK(cudaStreamSynchronize(h->s));
  h->have_prev = false;
  h->levels = 1;
  // the operator history of the given states, by the operator's own arithmetic
  h->ylev = 0;
  if (h->ydepth) {
    launch_apply_full(coef64(h, 0), h->x, nullptr, h->Y[0], h->s);
    h->ylev = 1;
  }
  if (xprev) {
    CKR(copy_in_dense(h, xprev, dof_of(h)));
    launch_pack(h->g, h->stage, h->xm, h->s);
    if (h->ydepth >= 2) {
      launch_apply_full(coef64(h, 0), h->xm, nullptr, h->Y[1], h->s);
      h->ylev = 2;
    }
    CK(cudaStreamSynchronize(h->s));
    h->have_prev = true;
    h->levels = 2;
  }
  h->t = t;
  h->step = step;
  return SD_OK;
}

int sd_get_history(sd_handle* h, double* xprev2) {
  if (!h || !xprev2) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  if (h->opt.extrapolate < 2 || h->levels < 3) return SD_E_STATE;
  launch_unpack(h->g, h->xmm, h->stage, h->s);
  CKR(copy_out(h, xprev2, h->stage, dof_of(h)));
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

int sd_set_history(sd_handle* h, const double* xprev2) {
  if (!h || !xprev2) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  if (h->opt.extrapolate < 2 || !h->have_prev || h->levels < 2) return SD_E_STATE;
  CKR(copy_in_dense(h, xprev2, dof_of(h)));
  launch_pack(h->g, h->stage, h->xmm, h->s);
  if (h->ydepth >= 3 && h->ylev >= 2) {
    launch_apply_full(coef64(h, 0), h->xmm, nullptr, h->Y[2], h->s);
    h->ylev = 3;
  }
  CK(cudaStreamSynchronize(h->s));
  h->levels = 3;
  return SD_OK;
}

int sd_apply(sd_handle* h, const double* x, double* y) {
  if (!h || !x || !y) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  const long long nd = dof_of(h);
  double* xin = h->V;                   // padded scratch in the Krylov slots
  double* yout = h->V + h->lenA;
  CKR(copy_in_dense(h, x, nd));
  launch_pack(h->g, h->stage, xin, h->s);
  launch_apply_full(coef64(h, 0), xin, nullptr, yout, h->s);
  launch_unpack(h->g, yout, h->stage, h->s);
  CKR(copy_out(h, y, h->stage, nd));
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

int sd_rhs(sd_handle* h, const double* xprev, double t, double* bout) {
  if (!h || !xprev || !bout) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  const long long nd = dof_of(h);
  double* xp = h->V;
  double* bb = h->V + h->lenA;
  CKR(copy_in_dense(h, xprev, nd));
  launch_pack(h->g, h->stage, xp, h->s);
  launch_rhs(h->g, h->opt.bc != SD_BC_MMS, h->g.h * h->g.h / h->dt, h->B0, h->B1, data_scale(h, t), xp, bb, xp, h->s);
  launch_unpack(h->g, bb, h->stage, h->s);
  CKR(copy_out(h, bout, h->stage, nd));
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

int sd_solve(sd_handle* h, const double* b, double* x, sd_step_info* info) {
  if (!h || !b || !x) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  t_pdl = h->opt.pdl;
  const long long nd = dof_of(h);
  h->ylev = 0;  // its residuals overwrite the newest operator-history entry
  // b and the iterate use the handle's b and a separate padded copy of x
  CKR(copy_in_dense(h, b, nd));
  launch_pack(h->g, h->stage, h->b, h->s);
  double* xs = h->B0;  // B0/B1 are rebuilt below; reuse B0 as the iterate
  CK(cudaStreamSynchronize(h->s));
  CKR(copy_in_dense(h, x, nd));
  launch_pack(h->g, h->stage, xs, h->s);
  sd_step_info si;
  std::memset(&si, 0, sizeof(si));
  CK(cudaEventRecord(h->e0, h->s));
  const int rc = fgmres(h, h->b, xs, &si);
  CK(cudaEventRecord(h->e1, h->s));
  launch_unpack(h->g, xs, h->stage, h->s);
  CKR(copy_out(h, x, h->stage, nd));
  CK(cudaEventSynchronize(h->e1));
  finish_block_residuals(h, &si);
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, h->e0, h->e1));
  si.ms = ms;
  // restore the manufactured-solution data that B0 held
  launch_mms_terms(coef64(h, 0), h->opt.bc, h->Klev[0], h->B0, h->B1, h->s);
  CK(cudaStreamSynchronize(h->s));
  if (info) *info = si;
  return rc;
}

int sd_sync(sd_handle* h) {
  if (!h) return SD_E_INVAL;
  CK(cudaStreamSynchronize(h->s));
  return SD_OK;
}

void sd_destroy(sd_handle* h) {
  if (!h) return;
  sdk::drop_batch_graph(h);  // a cached batch graph addresses the handle's memory
  if (h->s) cudaStreamSynchronize(h->s);
  for (auto& e : h->prof_ev)
    if (e) cudaEventDestroy(e);
  for (auto& gv : h->gexec)
    for (auto& ge : gv)
      if (ge) cudaGraphExecDestroy(ge);
  for (auto& sg : h->sg)
    if (sg.ex) cudaGraphExecDestroy(sg.ex);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->s2) {
    cudaStreamSynchronize(h->s2);
    cudaStreamDestroy(h->s2);
  }
  if (h->ar.base) cudaFree(h->ar.base);
  if (h->hflag) cudaFreeHost(h->hflag);
  if (h->e0) cudaEventDestroy(h->e0);
  if (h->e1) cudaEventDestroy(h->e1);
  if (h->own_stream && h->s) cudaStreamDestroy(h->s);
  delete h;
}

int sd_profile(sd_handle* h, int32_t kernel, int32_t enable) {
  if (!h) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  CK(cudaStreamSynchronize(h->s));
  prof_flush(h);
  if (h->prof_ev.empty()) {
    h->prof_ev.resize(4096);
    h->prof_bytes_pending.resize(2048);
    h->prof_flops_pending.resize(2048);
    for (auto& e : h->prof_ev) CK(cudaEventCreate(&e));
  }
  h->prof_id = enable ? kernel : -1;
  h->prof_ms = 0.0;
  h->prof_bytes = 0.0;
  h->prof_flops = 0.0;
  h->prof_launches = 0;
  return SD_OK;
}

int sd_profile_read(sd_handle* h, double* total_ms, int64_t* launches, double* bytes, double* flops) {
  if (!h) return SD_E_INVAL;
  std::lock_guard<std::mutex> lk(h->mtx);
  CK(cudaStreamSynchronize(h->s));
  prof_flush(h);
  if (total_ms) *total_ms = h->prof_ms;
  if (launches) *launches = h->prof_launches;
  if (bytes) *bytes = h->prof_bytes;
  if (flops) *flops = h->prof_flops;
  return SD_OK;
}

int64_t sd_launch_count(void) { return (int64_t)sdk::g_launch_count.load(); }

int64_t sd_struct_size(int32_t which) {
  switch (which) {
    case 0: return (int64_t)sizeof(sd_grid);
    case 1: return (int64_t)sizeof(sd_options);
    case 2: return (int64_t)sizeof(sd_step_info);
    case 3: return (int64_t)sizeof(sd_request);
    case 4: return (int64_t)sizeof(sd_result);
    default: return -1;
  }
}

const char* sd_strerror(int code) {
  switch (code) {
    case SD_OK: return "ok";
    case SD_PENDING: return "pending";
    case SD_E_INVAL: return "invalid argument";
    case SD_E_NOMEM: return "out of device memory or HBM budget";
    case SD_E_NOCONV: return "FGMRES did not reach rtol within max_iters";
    case SD_E_NUMERIC: return "NaN/Inf in the Krylov recurrence";
    case SD_E_TIMEOUT: return "timeout (reserved, not returned)";
    case SD_E_CUDA: return g_errmsg[0] ? g_errmsg : "CUDA error";
    case SD_E_STATE: return "unknown ticket or invalid state";
    default: return "unknown error";
  }
}

}  // extern "C"
