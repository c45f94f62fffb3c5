// sd_internal.cuh -- device data layout and launch wrappers of the GB300
// Stokes-Darcy solver (arXiv 2108.13229, Secs. 2 and 4).  Internal to the
// library; the public interface is include/sd.h.
//
// Layout of one level with n x n cells per subdomain (all fields share the
// row pitch P = roundup(n + 1, 8) elements, x fastest):
//   u    n     rows x P   vertical ff faces, i = 0..n   (i = 0, n: Dirichlet)
//   v    n + 1 rows x P   horizontal ff faces, i = 0..n-1 (j = 0: interface,
//                         j = n: Dirichlet)
//   p_ff n     rows x P   ff cell centres
//   p_pm n     rows x P   pm cell centres
// A whole-system vector is [u | v | p_ff | p_pm]; the velocity block V is the
// contiguous prefix [u | v]; the Darcy block D' is the suffix p_pm.  Padding
// entries are zero in every vector and no kernel writes them.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <type_traits>
#include <utility>
#include <vector>

namespace sdk {

// Programmatic dependent launch: when enabled for the calling host thread,
// kernels are launched with programmatic stream serialisation, so a grid's
// launch overlaps the drain of the previous grid.  Every kernel of this
// library starts with griddep_wait(), which returns once the previous grid
// has completed and its memory operations are visible, before the kernel
// touches global memory.  (An explicit early trigger for the next grid was
// measured and gave no gain.)
extern thread_local int t_pdl;
// Set by host threads that run instances side by side on their own streams
// (sd_solve_batch without lockstep): a launch of one instance then does not
// have the GPU to itself, which the tile shape of small levels assumes.
extern thread_local int t_conc;
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Lockstep batches (sd_solve_batch): instances whose buffers have identical
// layouts run in the same launches, one instance per blockIdx.z.  Every
// buffer of instance z is the same buffer of instance 0 moved by off[z]
// bytes (each instance's buffers come from one allocation laid out by the
// same plan), and act[z] == 0 makes the blocks of instance z return at once
// (instances that have converged wait for the others).  Kernels that take a
// Bat as their last parameter get it from launch_k: the calling host
// thread's t_bat, with the grid's z extent multiplied by t_bat_n.  With
// off == null (a single instance) nothing moves and blockIdx.z keeps any
// meaning the kernel gives it.
struct Bat {
  const long long* off;
  const int* act;
};
extern thread_local Bat t_bat;
extern thread_local int t_bat_n;
// set when a kernel without batch support is launched while t_bat is active
// (it would serve instance 0 only); the batch driver reports it
extern thread_local int t_bat_misuse;

// Byte offset of this block's instance; false if the instance is idle.
// Call after griddep_wait() (act is written by the host between launches).
__device__ __forceinline__ bool bat_enter(const Bat& b, long long& o) {
  o = 0;
  if (!b.off) return true;
  const int z = blockIdx.z;
  if (b.act && b.act[z] == 0) return false;
  o = b.off[z];
  return true;
}
template <typename P>
__device__ __forceinline__ P bsh(P p, long long o) {
  return p ? reinterpret_cast<P>(reinterpret_cast<uintptr_t>(p) + o) : p;
}

template <typename... Ts>
struct last_is_bat : std::false_type {};
template <typename T>
struct last_is_bat<T> : std::is_same<typename std::decay<T>::type, Bat> {};
template <typename T, typename U, typename... Ts>
struct last_is_bat<T, U, Ts...> : last_is_bat<U, Ts...> {};

template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), dim3 g, dim3 b, size_t smem, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = t_pdl ? 1 : 0;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if constexpr (last_is_bat<KArgs...>::value) {
    if (t_bat.off) cfg.gridDim.z *= (unsigned)t_bat_n;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)..., t_bat);
  } else {
    if (t_bat.off) t_bat_misuse = 1;
    cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
  }
}

// process-wide count of kernel launches made by this library (and the same
// count per host thread, used to size captured graphs)
extern std::atomic<long long> g_launch_count;
extern thread_local long long t_launch_count;
#define SD_COUNT(k) \
  (::sdk::t_launch_count += (k), ::sdk::g_launch_count.fetch_add((k), std::memory_order_relaxed))

struct Geom {
  int n;        // cells per side (porous medium; free-flow rows)
  int nx;       // free-flow cells across: n (square geometry) or 3n (the channel of Sec. 5)
  int iw;       // first free-flow column above the porous medium (0, or n in the channel)
  int P;        // row pitch in elements
  long long ou, ov, opf, opm, len;  // field offsets and whole-vector length
  long long lenV;                   // length of the velocity block [u | v]
  long long lenD;                   // length of the Darcy block
  double h;
};

// geo 0: free flow n x n over the porous medium n x n (Table 1); geo 1: the
// channel, free flow 3n x n whose floor's middle third is the interface
// (columns iw = n .. 2n-1), the rest of it a wall.  The porous-medium cells
// occupy columns 0 .. n-1 of their rows; the v face above pm cell i is the
// free-flow v face iw + i.
inline Geom make_geom(int n, int geo = 0) {
  Geom g;
  g.n = n;
  g.nx = geo == 1 ? 3 * n : n;
  g.iw = geo == 1 ? n : 0;
  g.P = ((g.nx + 1) + 7) / 8 * 8;
  g.ou = 0;
  g.ov = (long long)n * g.P;
  g.opf = (long long)(2 * n + 1) * g.P;
  g.opm = (long long)(3 * n + 1) * g.P;
  g.len = (long long)(4 * n + 1) * g.P;
  g.lenV = g.opf;
  g.lenD = (long long)n * g.P;
  g.h = 1.0 / n;
  return g;
}

// Coefficients of one level in precision T (Sec. 2 discretisation):
//   w[i]  = mu / (h + 2 beta_i), beta_i = mean sqrt(K) of the two pm cells
//           below interface u face i, over alpha_BJ (Eq. (6)); i = 1..n-1
//           (channel: u faces iw .. iw + n, the ends over one pm cell)
//   rg[i] = mu h^2 / (2 K_i) of the pm cell below v_Gamma face i (Eq. (5))
//           (channel: floor faces iw .. iw + n - 1)
//   Tx    n rows x P: TPFA transmissibility of the pm face left of cell i
//         (i = 0 and i = n: no-flow sides, 0)
//   Ty    (n+1) rows x P: face below cell row j (j = 0: Dirichlet bottom,
//         2K/mu; j = n: interface, 0 -- the flux there is h v_Gamma)
//         (pressure-Laplacian set: the same over its cx cells, with the
//         bottom faces Dirichlet only below the interface)
//   lat   1: the free-flow sides x = 0, 1 are traction sides (their u faces
//         are unknowns with half-control-volume rows; w[0] and w[n] are the
//         BJS coefficients of their interface corners); 0: Dirichlet sides
//   nx, iw free-flow cells across and the interface window [iw, iw + n) of
//         the free-flow floor faces (square geometry: nx = n, iw = 0)
//   cx    cells across of the cell block this set serves: n for the Darcy
//         set (and the Darcy rows of the whole operator), nx for the
//         pressure Laplacian of the free-flow cells
template <typename T>
struct Coef {
  int n, P;
  int nx, iw, cx;
  int lat;
  T h, mu, cm;  // cm = h^2 / dt
  const T* w;
  const T* rg;
  const T* Tx;
  const T* Ty;
  T d6, m1, m2;  // derived: cm + 6 mu (interior velocity diagonal), -mu, -2 mu
};

// fill the derived constants of a Coef from cm and mu
template <typename T>
inline void finish_coef(Coef<T>& c) {
  c.d6 = c.cm + T(6) * c.mu;
  c.m1 = -c.mu;
  c.m2 = T(-2) * c.mu;
}

// the coefficient arrays of a Coef moved to another instance of a batch
template <typename T>
__device__ __forceinline__ void bsh_coef(Coef<T>& c, long long o) {
  c.w = bsh(c.w, o);
  c.rg = bsh(c.rg, o);
  c.Tx = bsh(c.Tx, o);
  c.Ty = bsh(c.Ty, o);
}

// ---------------------------------------------------------------- sd_ops.cu
// setup
void launch_coarsen_K(const double* Kf, int nf, int Pf, double* Kc, int Pc, cudaStream_t s);
void launch_pack_K(const double* Kdense, int n, double* Kp, int P, cudaStream_t s);
void launch_fill_K(double* K, int cx, int n, int P, double v, cudaStream_t s);
// one coefficient set: Tx, Ty over cx x n cells of K (pitch P), the bottom
// faces Dirichlet over cells [b0, b1); w over u faces 0..nx and rg over floor
// faces 0..nx-1 from the top row of K, the interface over faces iw .. iw + n
template <typename T>
void launch_setup_coef(const double* Kp, int n, int cx, int P, double mu, double alpha, int lat, int xdir, int b0,
                       int b1, int nx, int iw, T* w, T* rg, T* Tx, T* Ty, cudaStream_t s);
template <typename T>
void launch_convert(const double* src, T* dst, long long len, cudaStream_t s, const double* rs = nullptr);
// top faces (row n) of the preconditioner's Darcy coefficients TyR: h^2 / d_i,
// d_i the diagonal of the v_Gamma row of floor face iw + i (Eq. (5)), the
// local Schur complement of the interface velocity eliminated through B'_1
// and C'_1 (nx: free-flow cells across; lat: traction sides)
void launch_darcy_schur_top(double* TyR, const double* w, const double* rg, int n, int nx, int iw, int P, double mu,
                            double cm, double h, int lat, cudaStream_t s);

// whole-system operator (FP64): y = A x  or  y = b - A x
void launch_apply_full(const Coef<double>& c, const double* x, const double* b, double* y, cudaStream_t s);
// r = b - A x together with its norms: sc[blk + 0..2] = ||r||^2 over the
// velocity, continuity and Darcy rows, sc[b2] = ||r||^2, and with with_b
// sc[bn] = ||b||^2 (partial: 4 * resid_norms_blocks(n) doubles of scratch).
// rh >= 0 (with with_b): when the device flag sc[rh] is set (launch_yhist),
// r holds A x already and the residual is b - r instead, with the same norms;
// the flag is cleared afterwards.  yo (may be null): A x is stored there too,
// formed by the operator's own arithmetic (as launch_apply_full's y = A x).
void launch_resid_norms(const Coef<double>& c, const double* x, const double* b, double* r, double* partial,
                        double* sc, int blk, int b2, int bn, int with_b, cudaStream_t s, int rh = -1,
                        double* yo = nullptr);
long long resid_norms_blocks(int nx, int n);
// y = A x together with the block partials of the first Gram-Schmidt pass's
// dot products of the Arnoldi step: partial[q * nblk + blk] for V_q . y, q <
// k <= apply_dots_max(), V_q = V + q vs in the whole-vector layout, nblk =
// resid_norms_blocks(n) (launch_reduce sums them)
void launch_apply_dots(const Coef<double>& c, const double* x, double* y, const double* V, long long vs, int k,
                       double* partial, cudaStream_t s);
int apply_dots_max();
// the free-flow rows of it (u, v, p_ff) with the porous-medium unknowns taken as zero;
// the Darcy rows of y are not written; vdir: the v_Gamma rows are identities
void launch_apply_ff(const Coef<double>& c, const double* x, const double* b, double* y, int vdir, cudaStream_t s);
// Darcy rows with the interface pressure prescribed over the half cell below Gamma
// (x, b, y: the p_pm block)
void launch_apply_pmd(const Coef<double>& c, const double* x, const double* b, double* y, cudaStream_t s);
// interface quantities of the free-flow-first order (ops in sd_ops.cu)
void launch_dn_iface(int op, const Coef<double>& c, const double* a, const double* b, const double* q, double* out,
                     cudaStream_t s);
// partitioned coupling: subdomain right-hand sides from the monolithic b.
//   pm: bs[p_pm] = b[p_pm] - h v on the cells below the interface (v: n values)
//   ff: bs[u, v, p_ff] = b + h p on the interface faces (p: n values, the pressure below)
void launch_dn_rhs_pm(const Geom& g, const double* b, const double* v, double* bs, cudaStream_t s);
void launch_dn_rhs_ff(const Geom& g, const double* b, const double* p, double* bs, cudaStream_t s);
// IQN-ILS update of the interface velocity (one CTA; see sd_krylov.cu)
struct IqnState {
  int n, qmax;
  double omega0;
  double* v;        // current input v_k, replaced by v_{k+1}
  double* p_prev;   // pressure and v~ of the previous evaluation, r_{k-1}
  double* vt_prev;
  double* r_prev;
  double* Vc;       // difference columns dr (qmax x ld), oldest first
  double* Wc;       // difference columns dv~
  double* Q;        // orthonormal basis of the Vc columns (modified Gram-Schmidt)
  double* R;        // upper triangle, column j at j * qmax
  double* scal;     // [0] k, [1] q, [2..5] |p - p_prev|^2, |p|^2, |v~ - v|^2, |v~|^2
  double* pG;       // free-flow-first order: the interface pressure and velocity of an evaluation
  double* vt;
  long long ld;     // column stride
};
void launch_iqn(const IqnState& st, const double* vt, const double* p, cudaStream_t s);

// right-hand side: b = mass * xprev + B0 + s1 * B1; also writes the Dirichlet
// values of b into x (so that the identity rows start exact); lat: traction sides
void launch_rhs(const Geom& g, int lat, double cm, const double* B0, const double* B1, double s1,
                const double* xprev, double* b, double* x, cudaStream_t s);
// boundary and source data: B0 (time-derivative part of the manufactured
// forcing), B1 (everything proportional to the time function s1 of
// launch_rhs: 1 + t for the manufactured cases bc 0, 1; the inflow pressure
// p_in(t) for the pressure-driven problem bc 2), and the exact state at time t
void launch_mms_terms(const Coef<double>& c, int bc, const double* Kp, double* B0, double* B1, cudaStream_t s);
void launch_mms_exact(const Geom& g, double mu, double t, double* x, cudaStream_t s);

// dense canonical layout <-> padded layout (whole-system vector)
void launch_pack(const Geom& g, const double* dense, double* padded, cudaStream_t s);
void launch_unpack(const Geom& g, const double* padded, double* dense, cudaStream_t s);

// block smoothers / residuals / transfers (T = float or double)
//   block V: velocity rows (u, v), identity on Dirichlet faces
//   block D: Darcy rows p_pm
// Chebyshev step: d = a d + c D^-1 (b - A x_in); x_out = x_in + d.
//   x_in == nullptr means x_in = 0;  a == 0 means d is not read.
//   ck (may be null): the same a, c in device memory (a = ck[0], c = ck[8]),
//   read instead in a lockstep batch, where they differ per instance.
template <typename T>
void launch_cheb_V(const Coef<T>& c, const T* x_in, const T* b, T* d, T* x_out, T a, T cc, const T* ck, int nbatch,
                   long long bstride, cudaStream_t s);
template <typename T>
void launch_cheb_D(const Coef<T>& c, const T* x_in, const T* b, T* d, T* x_out, T a, T cc, const T* ck, int nbatch,
                   long long bstride, cudaStream_t s);
// mode 0: r = b - A x (b == nullptr: r = -A x); 1: r = D^-1 A x; 2: r = A x
template <typename T>
void launch_resid_V(const Coef<T>& c, const T* x, const T* b, T* r, int jac, int nbatch, long long bstride,
                    cudaStream_t s);
template <typename T>
void launch_resid_D(const Coef<T>& c, const T* x, const T* b, T* r, int jac, int nbatch, long long bstride,
                    cudaStream_t s);
// coarse rhs = R r with R the transposed bilinear (V) / cell-sum (D) transfer;
// nxc, iwc: the coarse level's free-flow cells across and interface window
template <typename T>
void launch_restrict_V(int nf, int Pf, const T* r, int nc, int nxc, int iwc, int Pc, T* bc, int lat, cudaStream_t s);
template <typename T>
void launch_restrict_D(int nf, int Pf, const T* r, int nc, int Pc, T* bc, cudaStream_t s);
// cell blocks: bc = R (b - A x) with the cell-sum restriction, one pass
template <typename T>
void launch_resid_restrict_D(const Coef<T>& c, const T* x, const T* b, int nc, int Pc, T* bc, cudaStream_t s);
// x += P e (bilinear, staggered for V, cell-centred for D; xf: the fine
// cell block's cells across)
template <typename T>
void launch_prolong_V(int nf, int Pf, T* x, int nc, int nxc, int iwc, int Pc, const T* e, int lat, cudaStream_t s);
template <typename T>
void launch_prolong_D(int nf, int xf, int Pf, T* x, int nc, int Pc, const T* e, cudaStream_t s);

// Fused coarse V-cycle: levels c[0] (entry) .. c[nlev-1] (coarsest) in one
// CTA with shared-memory work vectors.  kind 0: velocity block, 1: cell block.
#define SD_CYC_MAXL 6
template <typename T>
struct CoarseCycle {
  int nlev, kind, m;
  int deg[SD_CYC_MAXL];  // Chebyshev steps per smoothing on each level
  Coef<T> c[SD_CYC_MAXL];
  T cha[SD_CYC_MAXL][8], chc[SD_CYC_MAXL][8];
  const T* cht[SD_CYC_MAXL];  // the same coefficients in device memory (a at 0..7, c at 8..15)
  const double* Ainv;
  const int* idx;
  const T* b_in;  // entry-level right-hand side (global, padded layout)
  T* x_out;       // entry-level result (global; valid entries written)
};
template <typename T>
size_t coarse_cycle_smem(const CoarseCycle<T>& q);
// returns -1 (nothing launched) if the levels need more shared memory than allowed
template <typename T>
int launch_coarse_cycle(const CoarseCycle<T>& q, cudaStream_t s);
// opt the kernel in to the large dynamic shared memory (once per device, before any capture)
template <typename T>
int prepare_coarse_cycle();

// Chebyshev step coefficients of one smoothing (ns <= 8 steps)
template <typename T>
struct ChebSteps {
  int ns;
  int rows;  // tiled smoothing: output rows per tile (8 or 16)
  int wave;  // FP32: 0, or the output rows per warp strip (8, 16, 32) of the register wavefront
  T a[8], c[8];
};
// Tiled smoothing: ns Chebyshev steps in one kernel, x_out = S(x_in + P ec)
// (x_in null: from zero; ec null: no prolongation).  FP32 only; returns -1
// (nothing launched) for ns > 4.  ct: the coefficients of cs in device
// memory (a at 0..7, c at 8..15), read instead in a lockstep batch.
template <typename T>
int launch_smooth_tile_D(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct,
                         const T* ec, int nc, int Pc, cudaStream_t s);
template <typename T>
int launch_smooth_tile_V(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct,
                         const T* ec, int nc, int Pc, cudaStream_t s);

// Pre-smoothing from zero that also forms the level's residual and restricts
// it to the coarse right-hand side bco (nc cells per side, pitch Pc): the
// smoothing of launch_smooth_tile_V/D plus the residual and restriction
// kernels of the level, the same values.  Returns -1 (nothing launched) for
// other tile heights, register-column tiles or an odd grid.
template <typename T>
int launch_smooth_tile_V_rr(const Coef<T>& c, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct, int nc,
                            int Pc, T* bco, cudaStream_t s);
template <typename T>
int launch_smooth_tile_D_rr(const Coef<T>& c, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct, int nc,
                            int Pc, T* bco, cudaStream_t s);

// Register-wavefront smoothing (sd_wave.cu): the same steps and result as
// the tiled kernels above, with cs.wave output rows per warp strip; returns -1
// (nothing launched) for ns > 4 or an unsupported strip height.
int launch_wave_V(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
                  const float* ct, const float* ec, int nc, int Pc, cudaStream_t s);
int launch_wave_D(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
                  const float* ct, const float* ec, int nc, int Pc, cudaStream_t s);

// preconditioner glue on the fine level (Sec. 4 block preconditioners):
//  entry: zpf = schur * r_pf + cmass * eP (eP: pressure-Laplacian solve, may be
//  null); rV = T(r_v - B zpf - B'_1 z_pm) (B omitted: use_B == 0; B'_1 only with
//  use_B1, reading the z_pm already in z)
//  rs (entry, mid, bgs_pff and launch_convert; null: 1): the device scale of
//  r, which is read as rs[0] r (the Krylov basis vector kept unnormalised)
template <typename T>
void launch_precond_entry(const Coef<double>& c, const double* r, double* z, double schur, const T* eP, double cmass,
                          int use_B, int use_B1, T* rV, cudaStream_t s, const double* rs = nullptr);
//  mid: z_v = double(eV); rD = T(r_pm - C'_1 z_v) (C'_1 omitted: use_C == 0; rD null: not written)
template <typename T>
void launch_precond_mid(const Coef<double>& c, const double* r, double* z, const T* eV, int use_C, T* rD,
                        cudaStream_t s, const double* rs = nullptr);
//  block Gauss-Seidel with identity on p_ff: z_pf = r_pf - C z_v
template <typename T>
void launch_precond_bgs_pff(const Coef<double>& c, const double* r, double* z, const T* eV, cudaStream_t s,
                            const double* rs = nullptr);
//  exit: z_pm = double(eD)
template <typename T>
void launch_precond_exit(const Coef<double>& c, double* z, const T* eD, cudaStream_t s);

// ------------------------------------------------------------- sd_krylov.cu
// number of blocks (= partial sums per dot product) for a vector of length len
int reduce_blocks(long long len);
// partial[i * ps + blk] = sum over the block's elements of V_i . w, i < k
//   cond (may be null): skipped when cond[0] == 0
void launch_mdot(const double* V, long long vstride, int k, const double* w, long long len, double* partial,
                 int ps, int nblk, const double* cond, cudaStream_t s);
// w -= sum_i coef[i] V_i, then partial dots of V_i . w (mode 1) or w . w (mode 2)
//   qs (may be null): scales of the V_i (kept unnormalised), folded into the coefficients
void launch_mupdate(const double* V, long long vstride, int k, const double* coef, double* w, long long len,
                    double* partial, int ps, int nblk, int mode, const double* cond, cudaStream_t s,
                    const double* qs = nullptr);
// out[i] = sum_b partial[i * ps + b], fixed order; cond (may be null): nothing
// when cond[0] == 0
//   qs (may be null): out[i] is multiplied by qs[i] (scales of unnormalised basis vectors)
void launch_reduce(const double* partial, int nblk, int k, int ps, double* out, const double* cond, cudaStream_t s,
                   const double* qs = nullptr);
// out[0] = sum_b partial[b] (= w'.w', the first Gram-Schmidt pass's projected
// w) and the re-orthogonalisation decision reo[0] = 1 when w'.w' < eta2
// (sum_{i < k1} h1[i]^2 + w'.w'), the right side being ||w||^2 before the
// projection (Pythagoras over the orthonormal basis), else 0
void launch_reduce_decide(const double* partial, int nblk, double* out, const double* h1, int k1, double eta2,
                          double* reo, cudaStream_t s);
// the operator history of the solved states, Y[i] = A x^{n-i} (depth 1..4
// entries): with use, r <- A x^0, the extrapolation of the given order (as
// launch_extrapolate's); then Y[i+1] <- Y[i]; rh[0] = use
void launch_yhist(double* const* Y, int depth, double* r, long long len, int order, int use, double* rh,
                  cudaStream_t s);
// history shift (x3 <- x_mm, x_mm <- x_m, x_m <- x; x3 may be null) and the
// extrapolation of the given order (1: linear, 2: quadratic, 3: cubic)
void launch_extrapolate(double* x, double* xm, double* xmm, double* x3, long long len, int order, cudaStream_t s);
// generic dot of two vectors: partials then reduce -> out[0]
void launch_dot(const double* a, const double* b, long long len, double* partial, int nblk, double* out,
                cudaStream_t s);
// y = alpha_dev[0]^p * x  (p = -1: divide by sqrt(alpha) ... see implementation)
void launch_scale_by(const double* x, double* y, long long len, const double* sdev, int mode, cudaStream_t s);
// (kdev, may be null: when given, k = kdev[0], read on the device; in a lockstep
// batch each instance's own)
void launch_axpy_multi(double* x, const double* Z, long long zstride, const double* ycoef, int k, long long len,
                       const double* kdev, cudaStream_t s);

//   the new column is hcol1 + hcol2 and its sub-diagonal sqrt(nrm2b) if reo is
//   null or reo[0] != 0 (second Gram-Schmidt pass done), else hcol1 and
//   sqrt(nrm2a) (hcol2 and nrm2b are then not read);
//   flag[5] = j + 1, the basis vectors of the cycle so far; vsc (may be null):
//   vsc[j + 1] = flag[1] = 1 / h_{j+1,j}, the scale of the new basis vector
void launch_givens(double* st, int j, int m, const double* hcol1, const double* hcol2, const double* nrm2a,
                   const double* nrm2b, const double* reo, double* flag, cudaStream_t s, double* vsc = nullptr);
void launch_backsolve(double* st, int k, int m, double* y, const double* kdev, cudaStream_t s);
// lockstep batches: out[z * count + t] = instance z's src[t]
void launch_gather_inst(const double* src, int count, double* out, cudaStream_t s);
//   vsc (may be null): vsc[0] = 1 / beta, the scale of the cycle's first basis vector
void launch_init_cycle(double* st, int m, const double* beta2, double* flag, cudaStream_t s, double* vsc = nullptr);

// device-side loop control of a whole FGMRES solve replayed as one graph
// (sd_krylov.cu).  ctl[C_TOL] tolerance on ||r||, ctl[C_BN] ||b||, the
// iteration, restart and second-pass counters, the status (0, or
// C_STAT_NUMERIC / C_STAT_NOCONV), the last true relative residual, the
// kernels run inside the graph's loops, the true residual before the last
// cycle and the residual a stagnating solve is accepted at (negative: never)
enum { C_TOL = 0, C_BN, C_ITER, C_REST, C_REO, C_STAT, C_REL, C_KERN, C_PREV, C_ACC, C_COUNT };
constexpr double C_STAT_NUMERIC = 1.0, C_STAT_NOCONV = 2.0;
struct CondSet {
  cudaGraphConditionalHandle c[32];  // c[j]: run Arnoldi step j (j >= 1)
  int n;                             // steps per cycle
};
void launch_solve_begin(const double* bn2, double rtol, double accept, double* ctl, cudaStream_t s);
void launch_restart_ctrl(const double* beta2, double* ctl, int max_iters, double kern,
                         cudaGraphConditionalHandle loop, cudaStream_t s);
void launch_cycle_head(const CondSet& cs, cudaStream_t s);
void launch_step_ctrl(double* flag, double* ctl, int max_iters, double kern, int has_next,
                      cudaGraphConditionalHandle next, cudaStream_t s);

// Device-side control of a lockstep group's solve inside one CUDA graph (the
// decisions of fgmres_lockstep, taken per instance on the device).  Each
// instance z's slots are its own ctl (ctl0 moved by off[z] bytes); act is the
// group's idle mask.  Beyond the single-solve slots: C_LIVE (the instance has
// not stopped), C_CYC (it takes part in the current cycle), C_NUMR (a NaN/Inf
// in the current cycle), and in instance 0's slots C_GCYC (the group's cycles
// so far).  One CTA each; they are not batched launches.
enum { C_LIVE = C_COUNT, C_CYC, C_NUMR, C_GCYC, C_GROUP_END };
//  act = 1 for every instance
void launch_grp_act_all(int* act, int B, cudaStream_t s);
//  tolerance rtol ||b|| from bn2 (each instance's ||b||^2), counters cleared, all live
void launch_grp_begin(const long long* off, int B, const double* bn2, double* ctl0, double rtol, cudaStream_t s);
//  after a true residual (b2: ||r||^2): per live instance stop (converged, NaN/Inf,
//  budget spent) or take part in a cycle (act = C_CYC); loop = any takes part;
//  cycles beyond max_cycles stop the group (a bound on the device loop)
void launch_grp_restart(const long long* off, int* act, int B, const double* b2, double* ctl0, int max_iters,
                        int max_cycles, double kern, cudaGraphConditionalHandle loop, cudaStream_t s);
//  after Arnoldi step j (flag0: each instance's flag): count it per active
//  instance, idle the ones that stop, and run step j + 1 if any goes on
void launch_grp_step(const long long* off, int* act, int B, const double* flag0, double* ctl0, int max_iters,
                     double kern, int has_next, cudaGraphConditionalHandle next, cudaStream_t s);
//  end of a cycle: a NaN/Inf stops the instance; act = C_CYC for the update of x
void launch_grp_cycle_end(const long long* off, int* act, int B, double* ctl0, double kern, cudaStream_t s);
//  act = C_LIVE (before the next true residual)
void launch_grp_live(const long long* off, int* act, int B, const double* ctl0, cudaStream_t s);

// dense coarse solve: x[idx[k]] = T(sum_l Ainv[k][l] * b[idx[l]])
template <typename T>
void launch_dense_solve(const double* Ainv, const int* idx, int m, const T* b, T* x, cudaStream_t s);
// Gauss-Jordan inverse with partial pivoting (setup only): A (m x m, destroyed),
// the inverse in W; fc: m doubles of scratch; counter: one int of scratch;
// *status = 0, or c + 1 for a zero pivot in column c
void launch_gj_inverse(double* A, double* W, int m, double* fc, int* status, int* counter, cudaStream_t s);
// identity batch in a padded layout: X[k * stride + idx[k]] = 1
void launch_identity_batch(double* X, long long stride, const int* idx, int m, cudaStream_t s);
void launch_gather_dense(const double* Y, long long stride, const int* idx, int m, double* A, cudaStream_t s);
void launch_fill(double* x, double v, long long len, cudaStream_t s);
void launch_hash_fill(double* x, long long len, unsigned seed, cudaStream_t s);

#ifdef SD_H
// ------------------------------------------------- lockstep batches (sd_api.cu)
// true if b can run in the same launches as a (same grid, mu, dt, options and
// buffer layout; no kernel timing active)
bool can_lockstep(const sd_handle* a, const sd_handle* b);
// nsteps implicit-Euler steps of count mutually compatible handles in lockstep
// on the first handle's stream; infos[i] (may be null) receives instance i's
// per-step information.  Returns the first non-OK step status.
int step_lockstep(sd_handle* const* hs, int count, int nsteps, sd_step_info* const* infos);
// Lockstep groups with every time step's solves of all groups in ONE graph
// launch: each group a branch whose restart loop and Arnoldi steps are decided
// on the device (WHILE / IF nodes, the k_grp_* kernels), the right-hand sides
// launched per group before it.  The last built graph is kept for the next
// call with the same groups.  groups[g] (mutually compatible handles)
// takes nsteps[g] steps; infos[g][i] (may be empty or null) receives handle
// i's per-step information.  Every instance's arithmetic is that of its solo
// run.  Returns the first non-OK step status.
int step_graph_batch(const std::vector<std::vector<sd_handle*>>& groups, const std::vector<int>& nsteps,
                     const std::vector<std::vector<sd_step_info*>>& infos);
// drop the cached batch graph if the handle is one of its instances
void drop_batch_graph(const sd_handle* h);
// cells per side of a handle's grid
int handle_grid(const sd_handle* h);
// unknowns of a handle's dense state vector
long long handle_dof(const sd_handle* h);
#endif

}  // namespace sdk
