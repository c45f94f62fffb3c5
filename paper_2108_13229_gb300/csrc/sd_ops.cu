// sd_ops.cu -- stencil kernels of the monolithic Stokes-Darcy solve
// (arXiv 2108.13229): the coupled operator of Eq. (9), the velocity block V
// and Darcy block D' used by the block preconditioners of Sec. 4, grid
// transfers of their geometric multigrid V-cycles, the preconditioner glue,
// coefficient setup and the implicit-Euler right-hand side.
//
// Discrete rows (every row integrated over its control volume, h = 1/n):
//  u face (i,j), 1<=i<=n-1:  (h^2/dt) u + 2mu(2u - uE - uW)          [normal stress]
//      + top corner:    mu(u - uN) - mu(vN,i - vN,i-1)   (j < n-1)
//                       2mu u                             (j = n-1, wall at h/2)
//      + bottom corner: mu(u - uS) + mu(v_i - v_i-1)      (j > 0)
//                       h w_i (2u + vG_i - vG_i-1)        (j = 0, BJS slip of Eq. (6)
//                                                          eliminated, w = mu/(h+2beta))
//      + h (p_i - p_i-1)                                  [block B]
//  v face (i,j), 1<=j<=n-1: symmetric to u, walls at x = 0, 1 at h/2.
//  v_Gamma face i (j = 0): half control volume [1, 1+h/2] (Eq. (5)):
//      (h^2/2dt + 2mu + mu h^2/(2K)) vG - 2mu v_i,1 + h p_ff - h p_pm[top]
//      + (h/2)(tau_W - tau_E), tau at interface corners from the BJS slip,
//        mu-only wall corners at x = 0, 1
//  p_ff cell: h (uE - uW + vN - vS)                       [Eq. (2), block C]
//  p_pm cell: sum_f T_f (p - p_nb) + h vG (top row)       [Eqs. (3),(4),(7); C'_1]
//  Dirichlet velocity faces: identity rows, eliminated from all other rows.
#include "sd_internal.cuh"
#include "sd_rows.cuh"

#include <math.h>

#include <type_traits>

namespace sdk {

static const int BX = 32, BY = 8;

static inline dim3 grid2(int nx, int ny) { return dim3((nx + BX - 1) / BX, (ny + BY - 1) / BY); }
// rows marched by one thread (measured on GB300): four consecutive rows help
// the FP64 operator from n = 512 and the cell-block kernels from n = 1024;
// the velocity-block kernels keep one row per thread (more blocks in flight)
static inline int rows_apply(int n) { return n >= 512 ? 4 : 1; }
static inline int rows_cell(int n) { return n >= 1024 ? 4 : 1; }
static inline int rows_vel(int) { return 1; }
static inline dim3 grid2R(int nx, int ny, int R) { return dim3((nx + BX - 1) / BX, (ny + BY * R - 1) / (BY * R)); }

// ------------------------------------------------------- whole operator (K1)
// What a launch of the operator forms on the side of y, as block partials in
// partial[q * nblocks + block]: with ND > 0 the dot products of y with the
// Krylov basis vectors V_q = V + q vs, q < ND (the first Gram-Schmidt pass of
// the Arnoldi step); with PS the residual's norms.
// skip (may be null): the launch returns at once when skip[0] != 0 (the
// step's first residual formed from the operator history, k_resid_hist).
// yo (YO: the residual form): A x itself is stored there too, formed by the
// operator's own arithmetic (the residual is then b - A x).
struct ApplySide {
  const double* V = nullptr;
  long long vs = 0;
  double* partial = nullptr;
  const double* skip = nullptr;
  double* yo = nullptr;
};

// dacc[q] += V_q[idx] * a, q < ND (one instantiation per count, as a
// masked-off FP64 instruction still takes its FP64-pipe cycles)
template <int ND>
__device__ __forceinline__ void side_dots(const ApplySide& sd, long long idx, double a, double* dacc) {
#pragma unroll
  for (int q = 0; q < ND; ++q) dacc[q] = fma(__ldg(sd.V + q * sd.vs + idx), a, dacc[q]);
}

// FF 1: the free-flow rows only (u, v, p_ff), with the porous-medium unknowns
// taken as zero and the Darcy rows not written (subdomain solve of the
// partitioned coupling); FF 2: the same with the v_Gamma rows replaced by
// identities (the interface velocity prescribed).
// Interior cells of the whole operator (FF 0): every row as one chain of
// fused multiply-adds from b (RES: y = b - A x) or from its first product (y
// = A x), its coefficients signed once per thread, so each stored matrix
// entry costs one FP64 instruction (the Darcy diagonal adds three).  The
// caller guarantees 2 <= i <= nx-2 and 1 <= j <= n-2, and with DARCY (the
// porous medium's rows at the same cell) i <= n-2.
// YO (with RES): every row is formed as A x, stored in sd.yo, and the
// residual is b - A x (the chain from b would give other roundings of A x).
template <bool RES, int PS, bool DARCY, int ND, bool YO = false>
__device__ __forceinline__ void apply_cell_interior(const Coef<double>& c, const double* __restrict__ u,
                                                    const double* __restrict__ v, const double* __restrict__ pf,
                                                    const double* __restrict__ pm, const double* __restrict__ b,
                                                    double* __restrict__ y, long long kc, long long nv,
                                                    long long npf, long long npm, double* acc,
                                                    const ApplySide& sd, double* dacc) {
  constexpr bool CH = RES && !YO;  // the chain starts from b
  const int P = c.P;
  const double sg = CH ? -1.0 : 1.0;
  const double kd = sg * c.d6, k2 = sg * c.m2, k1 = sg * c.m1, km = sg * c.mu, kh = sg * c.h;
  // the row's value a at index idx: y (and for YO, yo and the residual)
  auto emit = [&](long long idx, double a, int q) {
    double r = a;
    if constexpr (YO) {
      sd.yo[idx] = a;
      r = b[idx] - a;
    }
    y[idx] = r;
    side_dots<ND>(sd, idx, r, dacc);
    if (PS) acc[q] = fma(r, r, acc[q]);
    if (PS == 2) acc[3] = fma(b[idx], b[idx], acc[3]);
  };
  {  // u face: d6 u + m2 (uW + uE) + m1 (uN + vN + uS + vSW) + mu (vNW + vS) + h (pf - pfW)
    double a = CH ? fma(kd, u[kc], b[kc]) : kd * u[kc];
    a = fma(k2, u[kc - 1], a);
    a = fma(k2, u[kc + 1], a);
    a = fma(k1, u[kc + P], a);
    a = fma(k1, v[kc + P], a);
    a = fma(km, v[kc + P - 1], a);
    a = fma(k1, u[kc - P], a);
    a = fma(km, v[kc], a);
    a = fma(k1, v[kc - 1], a);
    a = fma(kh, pf[kc], a);
    a = fma(-kh, pf[kc - 1], a);
    emit(kc, a, 0);
  }
  {  // v face: d6 v + m2 (vS + vN) + m1 (vE + uE + vW + uWS) + mu (uES + uW) + h (pf - pfS)
    double a = CH ? fma(kd, v[kc], b[nv + kc]) : kd * v[kc];
    a = fma(k2, v[kc - P], a);
    a = fma(k2, v[kc + P], a);
    a = fma(k1, v[kc + 1], a);
    a = fma(k1, u[kc + 1], a);
    a = fma(km, u[kc + 1 - P], a);
    a = fma(k1, v[kc - 1], a);
    a = fma(km, u[kc], a);
    a = fma(k1, u[kc - P], a);
    a = fma(kh, pf[kc], a);
    a = fma(-kh, pf[kc - P], a);
    emit(nv + kc, a, 0);
  }
  {  // continuity: h (uE - uW + vN - vS)
    double a = CH ? fma(kh, u[kc + 1], b[npf + kc]) : kh * u[kc + 1];
    a = fma(-kh, u[kc], a);
    a = fma(kh, v[kc + P], a);
    a = fma(-kh, v[kc], a);
    emit(npf + kc, a, 1);
  }
  if (DARCY) {  // Darcy: (tw + te + ts + tn) p - tw pW - te pE - ts pS - tn pN
    const double tw = c.Tx[kc], te = c.Tx[kc + 1], ts = c.Ty[kc], tn = c.Ty[kc + P];
    const double kg = sg * ((tw + te) + (ts + tn));
    double a = CH ? fma(kg, pm[kc], b[npm + kc]) : kg * pm[kc];
    a = fma(-sg * tw, pm[kc - 1], a);
    a = fma(-sg * te, pm[kc + 1], a);
    a = fma(-sg * ts, pm[kc - P], a);
    a = fma(-sg * tn, pm[kc + P], a);
    emit(npm + kc, a, 2);
  }
}

// The operator's rows of this thread (i, j0 .. j0+R-1).  PS (with RES):
// acc[0..2] += the squared residuals of the velocity, continuity and Darcy
// rows; PS 2: also acc[3] += the squared right-hand side of every row.
template <int R, int FF, bool RES, int PS, int ND, bool YO = false>
__device__ __forceinline__ void apply_body(const Coef<double>& c, const double* __restrict__ x,
                                           const double* __restrict__ b, double* __restrict__ y, double* acc,
                                           const ApplySide& sd, double* dacc) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  const int n = c.n, nx = c.nx, P = c.P;
  if (i > nx) return;
  // a block none of whose points touches a boundary or the interface takes
  // the rows without their boundary cases (the same operations in the same
  // order for every interior point), so no masked FP64 work is issued; in
  // the channel a block beside the porous medium takes the free-flow rows
  // alone
  const int bi = blockIdx.x * blockDim.x, bj = blockIdx.y * blockDim.y * R;
  // (row 1 of the v faces reads the floor face below: in the channel an
  // interior block starts at row 2)
  const bool ff_in = bi >= 2 && bi + (int)blockDim.x - 1 <= nx - 2 && bj >= (c.iw ? 2 : 1) &&
                     bj + (int)blockDim.y * R - 1 <= n - 2;
  if (FF == 0 && ff_in && bi + (int)blockDim.x - 1 <= n - 2) {
    const long long nv = (long long)n * P, npf = (long long)(2 * n + 1) * P, npm = (long long)(3 * n + 1) * P;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      apply_cell_interior<RES, PS, true, ND, YO>(c, x, x + nv, x + npf, x + npm, b, y, (long long)(j0 + rr) * P + i,
                                                 nv, npf, npm, acc, sd, dacc);
    return;
  }
  if (FF == 0 && ff_in && bi >= n) {
    const long long nv = (long long)n * P, npf = (long long)(2 * n + 1) * P, npm = (long long)(3 * n + 1) * P;
#pragma unroll
    for (int rr = 0; rr < R; ++rr)
      apply_cell_interior<RES, PS, false, ND, YO>(c, x, x + nv, x + npf, x + npm, b, y, (long long)(j0 + rr) * P + i,
                                                  nv, npf, npm, acc, sd, dacc);
    return;
  }
  if (FF != 0 && ff_in && c.iw == 0) {
    const double h = c.h;
    const double* u = x;
    const double* v = x + (long long)n * P;
    const double* pf = x + (long long)(2 * n + 1) * P;
    const double* pm = x + (long long)(3 * n + 1) * P;
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int j = j0 + rr;
      const long long kc = (long long)j * P + i;
      {
        double off, dg;
        u_row<double, true>(c, u, v, i, j, true, off, dg);
        const double val = dg * u[kc] + off + h * (pf[kc] - pf[kc - 1]);
        y[kc] = b ? b[kc] - val : val;
      }
      const long long k = (long long)n * P + kc;
      {
        double off, dg;
        v_row<double, true>(c, u, v, i, j, true, off, dg);
        double val = dg * v[kc] + off;
        val += h * (pf[kc] - pf[kc - P]);
        y[k] = b ? b[k] - val : val;
      }
      double sd = -v[kc];
      sd += u[kc + 1];
      sd -= u[kc];
      sd += v[kc + P];
      const long long kp = (long long)(2 * n + 1) * P + kc;
      y[kp] = b ? b[kp] - h * sd : h * sd;
      if (FF) continue;
      double off, dg;
      d_row<double, true>(c, pm, i, j, true, off, dg);
      const double val = dg * pm[kc] + off;
      const long long km = (long long)(3 * n + 1) * P + kc;
      y[km] = b ? b[km] - val : val;
    }
    return;
  }
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j > c.n) break;
    const double h = c.h;
    const double* u = x;
    const double* v = x + (long long)n * P;
    const double* pf = x + (long long)(2 * n + 1) * P;
    const double* pm = x + (long long)(3 * n + 1) * P;
    if (j < n) {
      const long long k = (long long)j * P + i;
      double val;
      if ((i == 0 || i == nx) && !c.lat) {
        val = u[k];
      } else if (i == 0 || i == nx) {
        double off, dg;
        ub_row(c, u, v, i, j, true, off, dg);
        val = dg * u[k] + off + (i == 0 ? h * pf[k] : -h * pf[k - 1]);
      } else {
        double off, dg;
        u_row(c, u, v, i, j, true, off, dg);
        val = dg * u[k] + off + h * (pf[k] - pf[k - 1]);
      }
      {
        const double r_ = b ? b[k] - val : val;
        y[k] = r_;
        if constexpr (YO) sd.yo[k] = val;
        side_dots<ND>(sd, k, r_, dacc);
        if (PS) acc[0] = fma(r_, r_, acc[0]);
        if (PS == 2) acc[3] = fma(b[k], b[k], acc[3]);
      }
    }
    if (i < nx) {
      const long long kv = (long long)j * P + i;
      const long long k = (long long)n * P + kv;
      double val;
      if (j == n || (j == 0 && (FF == 2 || !on_gamma(c, i)))) {
        val = v[kv];
      } else {
        double off, dg;
        v_row(c, u, v, i, j, true, off, dg);
        val = dg * v[kv] + off;
        if (j > 0) val += h * (pf[kv] - pf[kv - P]);
        else if (FF) val += h * pf[i];
        else val += h * pf[i] - h * pm[(long long)(n - 1) * P + i - c.iw];
      }
      {
        const double r_ = b ? b[k] - val : val;
        y[k] = r_;
        if constexpr (YO) sd.yo[k] = val;
        side_dots<ND>(sd, k, r_, dacc);
        if (PS) acc[0] = fma(r_, r_, acc[0]);
        if (PS == 2) acc[3] = fma(b[k], b[k], acc[3]);
      }
    }
    if (i < nx && j < n) {
      const long long kc = (long long)j * P + i;
      // a floor face beside the interface is Dirichlet data (not an unknown)
      double s = (j > 0 || on_gamma(c, i)) ? -v[kc] : 0.0;
      if (c.lat || i + 1 <= nx - 1) s += u[kc + 1];
      if (c.lat || i >= 1) s -= u[kc];
      if (j + 1 <= n - 1) s += v[kc + P];
      const long long kp = (long long)(2 * n + 1) * P + kc;
      {
        const double val = h * s;
        {
          const double r_ = b ? b[kp] - val : val;
          y[kp] = r_;
          if constexpr (YO) sd.yo[kp] = val;
          side_dots<ND>(sd, kp, r_, dacc);
          if (PS) acc[1] = fma(r_, r_, acc[1]);
          if (PS == 2) acc[3] = fma(b[kp], b[kp], acc[3]);
        }
      }
    }
    if (!FF && i < n && j < n) {
      const long long kc = (long long)j * P + i;
      double off, dg;
      d_row(c, pm, i, j, true, off, dg);
      double val = dg * pm[kc] + off;
      if (j == n - 1) val += h * v[c.iw + i];
      const long long km = (long long)(3 * n + 1) * P + kc;
      {
        const double r_ = b ? b[km] - val : val;
        y[km] = r_;
        if constexpr (YO) sd.yo[km] = val;
        side_dots<ND>(sd, km, r_, dacc);
        if (PS) acc[2] = fma(r_, r_, acc[2]);
        if (PS == 2) acc[3] = fma(b[km], b[km], acc[3]);
      }
    }
  }
}

// PS / ND: the block's sums of acc (PS, apply_body's norms: q = 0..2, PS 2:
// 0..3) or dacc (ND: q < ND) in sd.partial[q * nblocks + block], in a fixed
// order, so repeated runs agree bit for bit.  FP64 adds are scarce on this
// part, so the block sums its values through shared memory with one warp per
// quantity (eight serial adds per lane, then five butterfly rounds) rather
// than a butterfly in every warp.
template <int R, int FF, bool RES, int PS = 0, int ND = 0, bool YO = false>
__global__ void __launch_bounds__(BX * BY, (PS || ND) ? 3 : 4)
    k_apply_full(Coef<double> c, const double* __restrict__ x, const double* __restrict__ b, double* __restrict__ y,
                 ApplySide sd, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    x = bsh(x, o);
    b = bsh(b, o);
    y = bsh(y, o);
    sd.V = bsh(sd.V, o);
    sd.partial = bsh(sd.partial, o);
    sd.skip = bsh(sd.skip, o);
    sd.yo = bsh(sd.yo, o);
  }
  if (sd.skip && sd.skip[0] != 0.0) return;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  double dacc[ND > 0 ? ND : 1];
#pragma unroll
  for (int q = 0; q < (ND > 0 ? ND : 1); ++q) dacc[q] = 0.0;
  apply_body<R, FF, RES, PS, ND, YO>(c, x, b, y, acc, sd, dacc);
  if constexpr (PS > 0 || ND > 0) {
    constexpr int NQ = PS == 2 ? 4 : PS == 1 ? 3 : ND;
    __shared__ double red[NQ][BX * BY];
    const int t = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
    for (int q = 0; q < NQ; ++q) red[q][t] = PS > 0 ? acc[q] : dacc[q];
    __syncthreads();
    const int wp = t >> 5, lane = t & 31;
    if (wp < NQ) {
      const double* r = red[wp] + lane * (BX * BY / 32);
      double v = r[0];
#pragma unroll
      for (int e = 1; e < BX * BY / 32; ++e) v += r[e];
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
      if (lane == 0) {
        const long long nbk = (long long)gridDim.x * gridDim.y;
        sd.partial[wp * nbk + (long long)blockIdx.y * gridDim.x + blockIdx.x] = v;
      }
    }
  }
}

// sc[blk + q] (q = 0..2) = the sums of squares of the residual's velocity,
// continuity and Darcy rows, sc[b2] = their total ((q0 + q1) + q2), and with
// with_b sc[bn] = the sum of squares of b; from the block partials of
// k_apply_full<.., PS>, each summed in a fixed order (every thread's partials
// loaded at once, then one warp per quantity).
__global__ void __launch_bounds__(256) k_reduce_resid(const double* __restrict__ partial, int nbk,
                                                      double* __restrict__ sc, int blk, int b2, int bn, int with_b,
                                                      int rh, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    partial = bsh(partial, o);
    sc = bsh(sc, o);
  }
  __shared__ double red[4][256];
  __shared__ double tot[4];
  const int t = threadIdx.x;
  const int nq = with_b ? 4 : 3;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = t; k < nbk; k += 256)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q < nq) v[q] += partial[(long long)q * nbk + k];
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][t] = v[q];
  __syncthreads();
  const int wp = t >> 5, lane = t & 31;
  if (wp < nq) {
    const double* r = red[wp] + lane * 8;
    double w = r[0];
#pragma unroll
    for (int e = 1; e < 8; ++e) w += r[e];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) w += __shfl_xor_sync(0xffffffffu, w, d);
    if (lane == 0) tot[wp] = w;
  }
  __syncthreads();
  if (t == 0) {
    sc[blk] = tot[0];
    sc[blk + 1] = tot[1];
    sc[blk + 2] = tot[2];
    sc[b2] = (tot[0] + tot[1]) + tot[2];
    if (with_b) sc[bn] = tot[3];
    if (rh >= 0) sc[rh] = 0.0;  // the history flag serves one residual
  }
}

// The step's first residual from the operator history (k_yhist): r = b - r,
// r holding A x^0 on entry (also stored in yo), with the norms of
// k_apply_full<.., PS 2> in its partial layout (the same grid and rows per
// thread, so k_reduce_resid sums whichever of the two ran); nothing unless
// run[0] != 0.  The Dirichlet faces' identity rows take A x^0 = x^0 from x
// itself, as the operator does: the right-hand side has put the new boundary
// data into x^0 there, which the extrapolated history does not know.
template <int R>
__global__ void __launch_bounds__(BX * BY) k_resid_hist(Coef<double> c, const double* __restrict__ x,
                                                        const double* __restrict__ b, double* __restrict__ r,
                                                        double* __restrict__ yo, double* __restrict__ partial,
                                                        const double* __restrict__ run, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    x = bsh(x, o);
    b = bsh(b, o);
    r = bsh(r, o);
    yo = bsh(yo, o);
    partial = bsh(partial, o);
    run = bsh(run, o);
  }
  if (run[0] == 0.0) return;
  const int n = c.n, nx = c.nx, P = c.P;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  const long long nv = (long long)n * P, npf = (long long)(2 * n + 1) * P, npm = (long long)(3 * n + 1) * P;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  auto put = [&](long long k, int q, bool ident) {
    const double ax = ident ? x[k] : r[k], bk = b[k], rk = bk - ax;
    yo[k] = ax;  // the newest entry of the history (a step solved by this residual alone keeps it)
    r[k] = rk;
    acc[q] = fma(rk, rk, acc[q]);
    acc[3] = fma(bk, bk, acc[3]);
  };
  if (i <= nx) {
#pragma unroll
    for (int rr = 0; rr < R; ++rr) {
      const int j = j0 + rr;
      if (j > n) break;
      const long long kc = (long long)j * P + i;
      if (j < n) put(kc, 0, (i == 0 || i == nx) && !c.lat);                    // u face
      if (i < nx) put(nv + kc, 0, j == n || (j == 0 && !on_gamma(c, i)));     // v face
      if (i < nx && j < n) put(npf + kc, 1, false);                            // continuity
      if (i < n && j < n) put(npm + kc, 2, false);                             // Darcy
    }
  }
  __shared__ double red[4][BX * BY];
  const int t = threadIdx.y * blockDim.x + threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) red[q][t] = acc[q];
  __syncthreads();
  const int wp = t >> 5, lane = t & 31;
  if (wp < 4) {
    const double* rq = red[wp] + lane * (BX * BY / 32);
    double v = rq[0];
#pragma unroll
    for (int e = 1; e < BX * BY / 32; ++e) v += rq[e];
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
    if (lane == 0) {
      const long long nbk = (long long)gridDim.x * gridDim.y;
      partial[wp * nbk + (long long)blockIdx.y * gridDim.x + blockIdx.x] = v;
    }
  }
}

template <int R, bool YO>
static void resid_go(const dim3& g, cudaStream_t s, const Coef<double>& c, const double* x, const double* b,
                     double* r, const ApplySide& sd, int with_b) {
  if (with_b) launch_k(k_apply_full<R, 0, true, 2, 0, YO>, g, dim3(BX, BY), 0, s, c, x, b, r, sd);
  else launch_k(k_apply_full<R, 0, true, 1, 0, YO>, g, dim3(BX, BY), 0, s, c, x, b, r, sd);
}

void launch_resid_norms(const Coef<double>& c, const double* x, const double* b, double* r, double* partial,
                        double* sc, int blk, int b2, int bn, int with_b, cudaStream_t s, int rh, double* yo) {
  SD_COUNT(rh >= 0 ? 3 : 2);
  const int R = rows_apply(c.n);
  const dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  ApplySide sd;
  sd.partial = partial;
  sd.skip = rh >= 0 ? sc + rh : nullptr;
  sd.yo = yo;
  if (rh >= 0) {
    if (R == 4) launch_k(k_resid_hist<4>, g, dim3(BX, BY), 0, s, c, x, b, r, yo, partial, (const double*)(sc + rh));
    else launch_k(k_resid_hist<1>, g, dim3(BX, BY), 0, s, c, x, b, r, yo, partial, (const double*)(sc + rh));
  }
  if (R == 4) {
    if (yo) resid_go<4, true>(g, s, c, x, b, r, sd, with_b);
    else resid_go<4, false>(g, s, c, x, b, r, sd, with_b);
  } else {
    if (yo) resid_go<1, true>(g, s, c, x, b, r, sd, with_b);
    else resid_go<1, false>(g, s, c, x, b, r, sd, with_b);
  }
  launch_k(k_reduce_resid, dim3(1), dim3(256), 0, s, (const double*)partial, (int)(g.x * g.y), sc, blk, b2, bn,
           with_b, rh);
}

// blocks of the operator's launch (partial sums per quantity of launch_resid_norms)
long long resid_norms_blocks(int nx, int n) {
  const dim3 g = grid2R(nx + 1, n + 1, rows_apply(n));
  return (long long)g.x * g.y;
}

// (at most four dot products: eight spilled registers at three blocks per SM)
int apply_dots_max() { return 4; }

void launch_apply_dots(const Coef<double>& c, const double* x, double* y, const double* V, long long vs, int k,
                       double* partial, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_apply(c.n);
  const dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  ApplySide sd;
  sd.V = V;
  sd.vs = vs;
  sd.partial = partial;
  const double* nb = nullptr;
  const dim3 bl(BX, BY);
  if (R == 4) {
    if (k == 1) launch_k(k_apply_full<4, 0, false, 0, 1>, g, bl, 0, s, c, x, nb, y, sd);
    else if (k == 2) launch_k(k_apply_full<4, 0, false, 0, 2>, g, bl, 0, s, c, x, nb, y, sd);
    else if (k == 3) launch_k(k_apply_full<4, 0, false, 0, 3>, g, bl, 0, s, c, x, nb, y, sd);
    else launch_k(k_apply_full<4, 0, false, 0, 4>, g, bl, 0, s, c, x, nb, y, sd);
  } else {
    if (k == 1) launch_k(k_apply_full<1, 0, false, 0, 1>, g, bl, 0, s, c, x, nb, y, sd);
    else if (k == 2) launch_k(k_apply_full<1, 0, false, 0, 2>, g, bl, 0, s, c, x, nb, y, sd);
    else if (k == 3) launch_k(k_apply_full<1, 0, false, 0, 3>, g, bl, 0, s, c, x, nb, y, sd);
    else launch_k(k_apply_full<1, 0, false, 0, 4>, g, bl, 0, s, c, x, nb, y, sd);
  }
}

void launch_apply_full(const Coef<double>& c, const double* x, const double* b, double* y, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_apply(c.n);
  const dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  if (R == 4) {
    if (b) launch_k(k_apply_full<4, 0, true>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
    else launch_k(k_apply_full<4, 0, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
  } else {
    if (b) launch_k(k_apply_full<1, 0, true>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
    else launch_k(k_apply_full<1, 0, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
  }
}

void launch_apply_ff(const Coef<double>& c, const double* x, const double* b, double* y, int vdir, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_apply(c.n);
  const dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  if (R == 4) {
    if (vdir) launch_k(k_apply_full<4, 2, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
    else launch_k(k_apply_full<4, 1, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
  } else {
    if (vdir) launch_k(k_apply_full<1, 2, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
    else launch_k(k_apply_full<1, 1, false>, g, dim3(BX, BY), 0, s, c, x, b, y, ApplySide());
  }
}

// Darcy rows with the interface pressure prescribed over the half cell below
// Gamma (transmissibility 2K/mu = h^2 / rg on the top row): the porous-medium
// solve of the order of Sec. 3.  x, b, y: the p_pm block (n rows x P).
__global__ void k_apply_pmd(Coef<double> c, const double* __restrict__ x, const double* __restrict__ b,
                            double* __restrict__ y) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n;
  if (i >= n || j >= n) return;
  const int k = j * c.P + i;
  double off, dg;
  d_row(c, x, i, j, true, off, dg);
  double val = dg * x[k] + off;
  if (j == n - 1) val += c.h * c.h / c.rg[i] * x[k];
  y[k] = b ? b[k] - val : val;
}

void launch_apply_pmd(const Coef<double>& c, const double* x, const double* b, double* y, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_apply_pmd, dim3(grid2(c.n, c.n)), dim3(dim3(BX, BY)), 0, s, c, x, b, y);
}

// Interface quantities of the order of Sec. 3 (n values each):
//  op 0: p_Gamma = (y_vG - rg v_G - b_vG) / h from the free-flow row y of the
//        v_Gamma faces (k_apply_full, FF 1), i.e. the normal stress balancing
//        the half control volume without the reconstruction term;
//  op 1: v~ = (h / rg) (p_top - p_Gamma), the Darcy velocity through Gamma;
//  op 2: bs[p_pm] = b[p_pm] (+ (h^2 / rg) p_Gamma on the top row);
//  op 3: bs[u, v, p_ff] = b with the v_Gamma rows replaced by v.
__global__ void k_dn_iface(int op, Coef<double> c, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ q, double* __restrict__ out) {
  griddep_wait();
  const int n = c.n, P = c.P;
  const double h = c.h;
  const long long ov = (long long)n * P, opm = (long long)(3 * n + 1) * P;
  const long long e0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
  if (op == 0) {
    for (long long i = e0; i < n; i += st) out[i] = (a[ov + i] - c.rg[i] * q[ov + i] - b[ov + i]) / h;
  } else if (op == 1) {
    for (long long i = e0; i < n; i += st) out[i] = h / c.rg[i] * (a[opm + (long long)(n - 1) * P + i] - q[i]);
  } else if (op == 2) {
    const long long len = (long long)n * P, top = (long long)(n - 1) * P;
    for (long long e = e0; e < len; e += st) {
      const long long i = e - top;
      out[opm + e] = (i >= 0 && i < n) ? b[opm + e] + h * h / c.rg[i] * q[i] : b[opm + e];
    }
  } else {
    for (long long e = e0; e < opm; e += st) {
      const long long i = e - ov;
      out[e] = (i >= 0 && i < n) ? q[i] : b[e];
    }
  }
}

void launch_dn_iface(int op, const Coef<double>& c, const double* a, const double* b, const double* q, double* out,
                     cudaStream_t s) {
  SD_COUNT(1);
  const long long work = op <= 1 ? c.n : (op == 2 ? (long long)c.n * c.P : (long long)(3 * c.n + 1) * c.P);
  const long long nb = (work + 255) / 256;
  launch_k(k_dn_iface, dim3((int)(nb < 152 * 16 ? nb : 152 * 16)), dim3(256), 0, s, op, c, a, b, q, out);
}

// --------------------------------------------- partitioned coupling (Sec. 3)
// Right-hand sides of the subdomain solves: the monolithic b with the other
// subdomain's unknowns moved over.  Darcy: the top cells' outflow h v_Gamma
// (block C'_1) with v_Gamma given.  Free flow: the -h p_pm term of the
// v_Gamma rows (block B'_1) with the pressure below the interface given.
__global__ void k_dn_rhs_pm(int n, int P, double h, const double* __restrict__ b, const double* __restrict__ v,
                            double* __restrict__ bs) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const long long k = (long long)(3 * n + 1) * P + (long long)j * P + i;
  bs[k] = j == n - 1 ? b[k] - h * v[i] : b[k];
}

__global__ void k_dn_rhs_ff(int n, int P, double h, const double* __restrict__ b, const double* __restrict__ p,
                            double* __restrict__ bs) {
  griddep_wait();
  const long long len = (long long)(3 * n + 1) * P, ov = (long long)n * P;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    const long long q = e - ov;
    bs[e] = (q >= 0 && q < n) ? b[e] + h * p[q] : b[e];
  }
}

void launch_dn_rhs_pm(const Geom& g, const double* b, const double* v, double* bs, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_dn_rhs_pm, dim3(grid2(g.n, g.n)), dim3(dim3(BX, BY)), 0, s, g.n, g.P, g.h, b, v, bs);
}

void launch_dn_rhs_ff(const Geom& g, const double* b, const double* p, double* bs, cudaStream_t s) {
  SD_COUNT(1);
  const long long len = (long long)(3 * g.n + 1) * g.P;
  const long long nb = (len + 255) / 256;
  launch_k(k_dn_rhs_ff, dim3((int)(nb < 152 * 16 ? nb : 152 * 16)), dim3(256), 0, s, g.n, g.P, g.h, b, p, bs);
}

// ------------------------------------------------------ block V smoothers
// One Chebyshev step at position (i, j) of the velocity block (u face (i,j)
// if j < n, v face (i,j) if i < nx).  Dirichlet faces take x = b exactly.
template <typename T, bool IN = false>
__device__ __forceinline__ void cheb_V_at2(const Coef<T>& c, const T* __restrict__ uin, const T* __restrict__ vin,
                                           const T* __restrict__ bu, const T* __restrict__ bv, T* __restrict__ du,
                                           T* __restrict__ dv, T* __restrict__ uout, T* __restrict__ vout, T a, T cc,
                                           int i, int j) {
  const int n = c.n, P = c.P;
  const bool rd = uin != nullptr;
  if (IN || j < n) {
    const int k = j * P + i;
    const bool side = !IN && (i == 0 || i == c.nx);
    if (side && !c.lat) {
      uout[k] = bu[k];
      du[k] = T(0);
    } else {
      T off, dg;
      if (side) ub_row(c, uin, vin, i, j, rd, off, dg);
      else u_row<T, IN>(c, uin, vin, i, j, rd, off, dg);
      const T xc = rd ? uin[k] : T(0);
      const T ad = a != T(0) ? a * du[k] : T(0);
      T dn, xn;
      cheb_point(bu[k], xc, off, dg, ad, cc, dn, xn);
      du[k] = dn;
      uout[k] = xn;
    }
  }
  if (IN || i < c.nx) {
    const int k = j * P + i;
    if (!IN && (j == n || (j == 0 && !on_gamma(c, i)))) {
      vout[k] = bv[k];
      dv[k] = T(0);
    } else {
      T off, dg;
      v_row<T, IN>(c, uin, vin, i, j, rd, off, dg);
      const T xc = rd ? vin[k] : T(0);
      const T ad = a != T(0) ? a * dv[k] : T(0);
      T dn, xn;
      cheb_point(bv[k], xc, off, dg, ad, cc, dn, xn);
      dv[k] = dn;
      vout[k] = xn;
    }
  }
}

template <typename T>
__device__ __forceinline__ void cheb_V_at(const Coef<T>& c, const T* __restrict__ xin, const T* __restrict__ b,
                                          T* __restrict__ d, T* __restrict__ xout, T a, T cc, int i, int j) {
  const long long nv = (long long)c.n * c.P;
  cheb_V_at2(c, xin, xin ? xin + nv : nullptr, b, b + nv, d, d + nv, xout, xout + nv, a, cc, i, j);
}

template <typename T, int R>
__global__ void k_cheb_V(Coef<T> c, const T* __restrict__ xin, const T* __restrict__ b, T* __restrict__ d,
                         T* __restrict__ xout, T a, T cc, const T* __restrict__ ck, long long bstride, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    d = bsh(d, o);
    xout = bsh(xout, o);
    if (ck) {
      a = bsh(ck, o)[0];
      cc = bsh(ck, o)[8];
    }
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i > c.nx) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j > c.n) break;
    const long long bo = (long long)blockIdx.z * bstride;
    cheb_V_at(c, xin ? xin + bo : nullptr, b + bo, d + bo, xout + bo, a, cc, i, j);
  }
}

template <typename T>
void launch_cheb_V(const Coef<T>& c, const T* x_in, const T* b, T* d, T* x_out, T a, T cc, const T* ck, int nbatch,
                   long long bstride, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_vel(c.n);
  dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  g.z = nbatch;
  if (R == 4) launch_k(k_cheb_V<T, 4>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x_in, b, d, x_out, a, cc, ck, bstride);
  else launch_k(k_cheb_V<T, 1>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x_in, b, d, x_out, a, cc, ck, bstride);
}

// r = b - V x (mode 0; b == nullptr: -V x), D^-1 V x (mode 1), V x (mode 2)
template <typename T>
__device__ __forceinline__ void resid_V_at(const Coef<T>& c, const T* __restrict__ x, const T* __restrict__ b,
                                           T* __restrict__ r, int jac, int i, int j) {
  const int n = c.n, nx = c.nx, P = c.P;
  const T* u = x;
  const T* v = x + (long long)n * P;
  if (j < n) {
    const int k = j * P + i;
    T ax, dg = T(1);
    if ((i == 0 || i == nx) && !c.lat) {
      ax = x[k];
    } else {
      T off;
      if (i == 0 || i == nx) ub_row(c, u, v, i, j, true, off, dg);
      else u_row(c, u, v, i, j, true, off, dg);
      ax = dg * x[k] + off;
    }
    r[k] = jac == 1 ? ax / dg : (jac == 2 ? ax : (b ? b[k] - ax : -ax));
  }
  if (i < nx) {
    const int k = n * P + j * P + i;
    T ax, dg = T(1);
    if (j == n || (j == 0 && !on_gamma(c, i))) {
      ax = x[k];
    } else {
      T off;
      v_row(c, u, v, i, j, true, off, dg);
      ax = dg * x[k] + off;
    }
    r[k] = jac == 1 ? ax / dg : (jac == 2 ? ax : (b ? b[k] - ax : -ax));
  }
}

template <typename T, int R>
__global__ void k_resid_V(Coef<T> c, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, int jac,
                          long long bstride, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    x = bsh(x, o);
    b = bsh(b, o);
    r = bsh(r, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i > c.nx) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j > c.n) break;
    const long long bo = (long long)blockIdx.z * bstride;
    resid_V_at(c, x + bo, b ? b + bo : nullptr, r + bo, jac, i, j);
  }
}

template <typename T>
void launch_resid_V(const Coef<T>& c, const T* x, const T* b, T* r, int jac, int nbatch, long long bstride,
                    cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_vel(c.n);
  dim3 g = grid2R(c.nx + 1, c.n + 1, R);
  g.z = nbatch;
  if (R == 4) launch_k(k_resid_V<T, 4>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x, b, r, jac, bstride);
  else launch_k(k_resid_V<T, 1>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x, b, r, jac, bstride);
}

// ------------------------------------------------------ block D' smoothers
template <typename T, bool IN = false>
__device__ __forceinline__ void cheb_D_at(const Coef<T>& c, const T* __restrict__ xin, const T* __restrict__ b,
                                          T* __restrict__ d, T* __restrict__ xout, T a, T cc, int i, int j) {
  const int k = j * c.P + i;
  const bool rd = xin != nullptr;
  T off, dg;
  d_row<T, IN>(c, xin, i, j, rd, off, dg);
  const T xc = rd ? xin[k] : T(0);
  const T ad = a != T(0) ? a * d[k] : T(0);
  T dn, xn;
  cheb_point(b[k], xc, off, dg, ad, cc, dn, xn);
  d[k] = dn;
  xout[k] = xn;
}

template <typename T, int R>
__global__ void k_cheb_D(Coef<T> c, const T* __restrict__ xin, const T* __restrict__ b, T* __restrict__ d,
                         T* __restrict__ xout, T a, T cc, const T* __restrict__ ck, long long bstride, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    d = bsh(d, o);
    xout = bsh(xout, o);
    if (ck) {
      a = bsh(ck, o)[0];
      cc = bsh(ck, o)[8];
    }
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i >= c.cx) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j >= c.n) break;
    const long long bo = (long long)blockIdx.z * bstride;
    cheb_D_at(c, xin ? xin + bo : nullptr, b + bo, d + bo, xout + bo, a, cc, i, j);
  }
}

template <typename T>
void launch_cheb_D(const Coef<T>& c, const T* x_in, const T* b, T* d, T* x_out, T a, T cc, const T* ck, int nbatch,
                   long long bstride, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_cell(c.n);
  dim3 g = grid2R(c.cx, c.n, R);
  g.z = nbatch;
  if (R == 4) launch_k(k_cheb_D<T, 4>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x_in, b, d, x_out, a, cc, ck, bstride);
  else launch_k(k_cheb_D<T, 1>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x_in, b, d, x_out, a, cc, ck, bstride);
}

template <typename T>
__device__ __forceinline__ void resid_D_at(const Coef<T>& c, const T* __restrict__ x, const T* __restrict__ b,
                                           T* __restrict__ r, int jac, int i, int j) {
  const int k = j * c.P + i;
  T off, dg;
  d_row(c, x, i, j, true, off, dg);
  const T ax = dg * x[k] + off;
  r[k] = jac == 1 ? ax / dg : (jac == 2 ? ax : (b ? b[k] - ax : -ax));
}

template <typename T, int R>
__global__ void k_resid_D(Coef<T> c, const T* __restrict__ x, const T* __restrict__ b, T* __restrict__ r, int jac,
                          long long bstride, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    x = bsh(x, o);
    b = bsh(b, o);
    r = bsh(r, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i >= c.cx) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j >= c.n) break;
    const long long bo = (long long)blockIdx.z * bstride;
    resid_D_at(c, x + bo, b ? b + bo : nullptr, r + bo, jac, i, j);
  }
}

template <typename T>
void launch_resid_D(const Coef<T>& c, const T* x, const T* b, T* r, int jac, int nbatch, long long bstride,
                    cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_cell(c.n);
  dim3 g = grid2R(c.cx, c.n, R);
  g.z = nbatch;
  if (R == 4) launch_k(k_resid_D<T, 4>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x, b, r, jac, bstride);
  else launch_k(k_resid_D<T, 1>, dim3(g), dim3(dim3(BX, BY)), 0, s, c, x, b, r, jac, bstride);
}

// ------------------------------------------------------------ transfers
// (prolongation values: sd_rows.cuh)
// coarse faces (I, J) of the velocity block from the fine residual, its u and
// v parts at ru, rv (row pitch Pf); the coarse level has nxc free-flow cells
// across and its interface under floor faces iwc .. iwc + nc - 1 (the
// transpose of prolong_u_val / prolong_v_val with their ghosts)
template <typename T>
__device__ __forceinline__ void restrict_V_at2(const T* __restrict__ ru, const T* __restrict__ rv, int Pf, int nc,
                                               int nxc, int iwc, int Pc, T* __restrict__ bc, int I, int J, int lat) {
  if (J < nc) {
    T s = T(0);
    // fine row 0 below coarse row 0: the ghost is +row 0 over the interface
    // (weights 3/4 + 1/4) and -row 0 over a wall (3/4 - 1/4)
    const T w00 = (I >= iwc && I <= iwc + nc) ? T(1) : T(0.5);
    if (lat && (I == 0 || I == nxc)) {  // traction side face: the one-sided transpose of the prolongation
      int rows[4];
      T wy[4];
      rows[0] = 2 * J - 1; wy[0] = J >= 1 ? T(0.25) : T(0);
      rows[1] = 2 * J;     wy[1] = J == 0 ? w00 : T(0.75);
      rows[2] = 2 * J + 1; wy[2] = J == nc - 1 ? T(0.5) : T(0.75);
      rows[3] = 2 * J + 2; wy[3] = J <= nc - 2 ? T(0.25) : T(0);
      const int ii = 2 * I, in = I == 0 ? 1 : 2 * I - 1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (wy[q] == T(0)) continue;
        const T* row = ru + (long long)rows[q] * Pf;
        s += wy[q] * (row[ii] + T(0.5) * row[in]);
      }
    } else if (I > 0 && I < nxc) {
      int rows[4];
      T wy[4];
      rows[0] = 2 * J - 1; wy[0] = J >= 1 ? T(0.25) : T(0);
      rows[1] = 2 * J;     wy[1] = J == 0 ? w00 : T(0.75);
      rows[2] = 2 * J + 1; wy[2] = J == nc - 1 ? T(0.5) : T(0.75);
      rows[3] = 2 * J + 2; wy[3] = J <= nc - 2 ? T(0.25) : T(0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (wy[q] == T(0)) continue;
        const T* row = ru + (long long)rows[q] * Pf;
        s += wy[q] * (row[2 * I] + T(0.5) * (row[2 * I - 1] + row[2 * I + 1]));
      }
    }
    bc[(long long)J * Pc + I] = s;
  }
  if (I < nxc) {
    T s = T(0);
    // a coarse floor face beside the interface is Dirichlet (right-hand side 0)
    if (J < nc && !(J == 0 && iwc > 0 && (I < iwc || I >= iwc + nc))) {
      int cols[4];
      T wx[4];
      cols[0] = 2 * I - 1; wx[0] = I >= 1 ? T(0.25) : T(0);
      cols[1] = 2 * I;     wx[1] = I == 0 ? T(0.5) : T(0.75);
      cols[2] = 2 * I + 1; wx[2] = I == nxc - 1 ? T(0.5) : T(0.75);
      cols[3] = 2 * I + 2; wx[3] = I <= nxc - 2 ? T(0.25) : T(0);
      const T* r0 = rv + (long long)(2 * J) * Pf;
      const T* r1 = rv + (long long)(2 * J + 1) * Pf;
      const T* rm = J >= 1 ? rv + (long long)(2 * J - 1) * Pf : nullptr;
      // fine floor faces beside the interface take no prolongation
      const int f0 = 2 * iwc, f1 = 2 * (iwc + nc);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (wx[q] == T(0)) continue;
        const int ci = cols[q];
        const T r00 = (J > 0 || iwc == 0 || (ci >= f0 && ci < f1)) ? r0[ci] : T(0);
        T t = r00 + T(0.5) * r1[ci];
        if (rm) t += T(0.5) * rm[ci];
        s += wx[q] * t;
      }
    }
    bc[(long long)nc * Pc + (long long)J * Pc + I] = s;
  }
}

template <typename T>
__device__ __forceinline__ void restrict_V_at(int nf, int Pf, const T* __restrict__ r, int nc, int nxc, int iwc,
                                              int Pc, T* __restrict__ bc, int I, int J, int lat = 0) {
  restrict_V_at2(r, r + (long long)nf * Pf, Pf, nc, nxc, iwc, Pc, bc, I, J, lat);
}

template <typename T>
__global__ void k_restrict_V(int nf, int Pf, const T* __restrict__ r, int nc, int nxc, int iwc, int Pc,
                             T* __restrict__ bc, int lat, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    r = bsh(r, o);
    bc = bsh(bc, o);
  }
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I > nxc || J > nc) return;
  restrict_V_at(nf, Pf, r, nc, nxc, iwc, Pc, bc, I, J, lat);
}

template <typename T>
void launch_restrict_V(int nf, int Pf, const T* r, int nc, int nxc, int iwc, int Pc, T* bc, int lat, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_restrict_V<T>, dim3(grid2(nxc + 1, nc + 1)), dim3(dim3(BX, BY)), 0, s, nf, Pf, r, nc, nxc, iwc, Pc, bc,
           lat);
}

template <typename T>
__device__ __forceinline__ void restrict_D_at(int Pf, const T* __restrict__ r, int Pc, T* __restrict__ bc, int I,
                                              int J) {
  const T* r0 = r + (long long)(2 * J) * Pf + 2 * I;
  bc[(long long)J * Pc + I] = (r0[0] + r0[1]) + (r0[Pf] + r0[Pf + 1]);
}

template <typename T>
__global__ void k_restrict_D(int nf, int Pf, const T* __restrict__ r, int nc, int Pc, T* __restrict__ bc, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    r = bsh(r, o);
    bc = bsh(bc, o);
  }
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= nc || J >= nc) return;
  restrict_D_at(Pf, r, Pc, bc, I, J);
}

template <typename T>
void launch_restrict_D(int nf, int Pf, const T* r, int nc, int Pc, T* bc, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_restrict_D<T>, dim3(grid2(nc, nc)), dim3(dim3(BX, BY)), 0, s, nf, Pf, r, nc, Pc, bc);
}

// Cell blocks: b_c(I, J) = sum of the residuals b - A x of the four fine
// cells of coarse cell (I, J) (residual and cell-sum restriction in one pass).
template <typename T>
__global__ void k_resid_restrict_D(Coef<T> c, const T* __restrict__ x, const T* __restrict__ b, int nc, int Pc,
                                   T* __restrict__ bc, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    x = bsh(x, o);
    b = bsh(b, o);
    bc = bsh(bc, o);
  }
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I >= c.cx / 2 || J >= nc) return;
  T r[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = 2 * I + (q & 1), j = 2 * J + (q >> 1);
    const long long k = (long long)j * c.P + i;
    T off, dg;
    d_row(c, x, i, j, true, off, dg);
    r[q] = b[k] - (dg * x[k] + off);
  }
  bc[(long long)J * Pc + I] = (r[0] + r[1]) + (r[2] + r[3]);
}

template <typename T>
void launch_resid_restrict_D(const Coef<T>& c, const T* x, const T* b, int nc, int Pc, T* bc, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_resid_restrict_D<T>, dim3(grid2(c.cx / 2, nc)), dim3(dim3(BX, BY)), 0, s, c, x, b, nc, Pc, bc);
}

// (fine faces: u i = 0 .. 2 nxc, v i < 2 nxc; the Dirichlet faces, the floor
// faces beside the interface among them, take no increment)
template <typename T>
__device__ __forceinline__ void prolong_V_at(int nf, int Pf, T* __restrict__ x, int nc, int nxc, int iwc, int Pc,
                                             const T* __restrict__ e, int i, int j, int lat = 0) {
  const T* eu = e;
  const T* ev = e + (long long)nc * Pc;
  const int nxf = 2 * nxc;
  if (j < nf && (lat || (i > 0 && i < nxf)))
    x[(long long)j * Pf + i] += prolong_u_val(eu, nc, nxc, iwc, Pc, i, j, lat);
  if (i < nxf && j < nf && !(j == 0 && iwc > 0 && (i < 2 * iwc || i >= 2 * (iwc + nc))))
    x[(long long)nf * Pf + (long long)j * Pf + i] += prolong_v_val(ev, nc, nxc, iwc, Pc, i, j);
}

template <typename T, int R>
__global__ void k_prolong_V(int nf, int Pf, T* __restrict__ x, int nc, int nxc, int iwc, int Pc,
                            const T* __restrict__ e, int lat, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    x = bsh(x, o);
    e = bsh(e, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i > 2 * nxc) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j > nf) break;
    prolong_V_at(nf, Pf, x, nc, nxc, iwc, Pc, e, i, j, lat);
  }
}

template <typename T>
void launch_prolong_V(int nf, int Pf, T* x, int nc, int nxc, int iwc, int Pc, const T* e, int lat, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_vel(nf);
  if (R == 4)
    launch_k(k_prolong_V<T, 4>, dim3(grid2R(2 * nxc + 1, nf + 1, 4)), dim3(dim3(BX, BY)), 0, s, nf, Pf, x, nc, nxc,
             iwc, Pc, e, lat);
  else
    launch_k(k_prolong_V<T, 1>, dim3(grid2R(2 * nxc + 1, nf + 1, 1)), dim3(dim3(BX, BY)), 0, s, nf, Pf, x, nc, nxc,
             iwc, Pc, e, lat);
}

template <typename T>
__device__ __forceinline__ void prolong_D_at(int Pf, T* __restrict__ x, int nc, int ncx, int Pc,
                                             const T* __restrict__ e, int i, int j) {
  x[(long long)j * Pf + i] += prolong_D_val(e, nc, ncx, Pc, i, j);
}

template <typename T, int R>
__global__ void k_prolong_D(int nf, int xf, int Pf, T* __restrict__ x, int nc, int Pc, const T* __restrict__ e,
                            Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    x = bsh(x, o);
    e = bsh(e, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j0 = (blockIdx.y * blockDim.y + threadIdx.y) * R;
  if (i >= xf) return;
#pragma unroll
  for (int rr = 0; rr < R; ++rr) {
    const int j = j0 + rr;
    if (j >= nf) break;
    prolong_D_at(Pf, x, nc, xf / 2, Pc, e, i, j);
  }
}

template <typename T>
void launch_prolong_D(int nf, int xf, int Pf, T* x, int nc, int Pc, const T* e, cudaStream_t s) {
  SD_COUNT(1);
  const int R = rows_cell(nf);
  if (R == 4)
    launch_k(k_prolong_D<T, 4>, dim3(grid2R(xf, nf, 4)), dim3(dim3(BX, BY)), 0, s, nf, xf, Pf, x, nc, Pc, e);
  else
    launch_k(k_prolong_D<T, 1>, dim3(grid2R(xf, nf, 1)), dim3(dim3(BX, BY)), 0, s, nf, xf, Pf, x, nc, Pc, e);
}

// ------------------------------------------- tiled (temporally blocked) smoothing
// NS Chebyshev steps in one kernel.  Each block loads an output tile of
// TLX x TLY positions plus a halo of NS (one per step: every step reaches one
// neighbour) into shared memory, with x_in optionally increased by the
// prolongation of a coarse correction, runs the NS steps there (the computed
// region shrinks by one per step), and writes only its output tile.  Each
// point's arithmetic is that of the per-step kernels, in the same order, so
// the result is bitwise the same; only the global traffic and the launches
// of the intermediate steps disappear.
static const int TLX = 32, TLT = 256;  // tile width and threads; the height TLY is a template parameter

// Prolongation inside the tiled smoothers.  The coarse correction around a
// tile is staged once in shared memory as the values cu_at / cv_at / cd_at
// return (ghosts and mirrors included) on a CX x CY coarse window whose
// corner is (I0, J0); every halo point's increment is then formed from that
// window with the operations of prolong_u_val / prolong_v_val /
// prolong_D_val in the same order, so it is bitwise the same.  (Formed from
// global memory, the increments took as many instructions as the three
// smoothing steps of a tile.)
template <typename T>
__device__ __forceinline__ T prolong_u_sm(const T* __restrict__ s, int CX, int I0, int J0, int i, int j) {
  const int J = j >> 1, Jn = (j & 1) ? J + 1 : J - 1;
  const int I = i >> 1;
  const T* r0 = s + (J - J0) * CX + (I - I0);
  const T* r1 = s + (Jn - J0) * CX + (I - I0);
  T cy0, cy1;
  if (i & 1) {
    cy0 = T(0.5) * (r0[0] + r0[1]);
    cy1 = T(0.5) * (r1[0] + r1[1]);
  } else {
    cy0 = r0[0];
    cy1 = r1[0];
  }
  return T(0.75) * cy0 + T(0.25) * cy1;
}
template <typename T>
__device__ __forceinline__ T prolong_v_sm(const T* __restrict__ s, int CX, int I0, int J0, int i, int j) {
  const int I = i >> 1, In = (i & 1) ? I + 1 : I - 1;
  const int J = j >> 1;
  const T* r0 = s + (J - J0) * CX;
  T cx0, cx1;
  if (j & 1) {
    cx0 = T(0.5) * (r0[I - I0] + r0[CX + I - I0]);
    cx1 = T(0.5) * (r0[In - I0] + r0[CX + In - I0]);
  } else {
    cx0 = r0[I - I0];
    cx1 = r0[In - I0];
  }
  return T(0.75) * cx0 + T(0.25) * cx1;
}
template <typename T>
__device__ __forceinline__ T prolong_D_sm(const T* __restrict__ s, int CX, int I0, int J0, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  const int In = (i & 1) ? I + 1 : I - 1, Jn = (j & 1) ? J + 1 : J - 1;
  const T* r0 = s + (J - J0) * CX - I0;
  const T* r1 = s + (Jn - J0) * CX - I0;
  return T(0.5625) * r0[I] + T(0.1875) * (r0[In] + r1[I]) + T(0.0625) * r1[In];
}

// RR (pre-smoothing from zero only): the tile also forms the residual of its
// output cells (x smoothed on a halo of NS + 1 for that) and sums it over the
// 2 x 2 children of each coarse cell it covers into bco (nc x nc, pitch Pc):
// k_resid_restrict_D's work and arithmetic, without its launch.
template <typename T, int NS, int TLY, bool BT, bool RR = false, int NT = TLT>
__global__ void __launch_bounds__(NT, NT > TLT ? 2 : (TLY <= 8 ? 8 : 4))
    k_smooth_tile_D(Coef<T> c, const T* __restrict__ xin, const T* __restrict__ b, T* __restrict__ xout,
                    ChebSteps<T> cs, const T* __restrict__ ct, const T* __restrict__ ec, int nc, int Pc,
                    T* __restrict__ bco, Bat bt) {
  griddep_wait();
  // a separate instantiation for lockstep batches keeps the single-instance
  // kernel's coefficients in the parameter space
  if constexpr (BT) {
    long long o;
    if (!bat_enter(bt, o)) return;
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    xout = bsh(xout, o);
    ec = bsh(ec, o);
    bco = bsh(bco, o);
    if (ct) {
      const T* q = bsh(ct, o);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        cs.a[s] = q[s];
        cs.c[s] = q[8 + s];
      }
    }
  }
  constexpr int H = RR ? NS + 1 : NS, EX = TLX + 2 * H, EY = TLY + 2 * H, SP = EX + 1, SR = EY + 1;
  constexpr int CX = SP / 2 + 4, CY = SR / 2 + 4;  // coarse window of the prolongation
  __shared__ T sb[SR * SP], sx0[SR * SP], sx1[SR * SP], sd[SR * SP], sTx[SR * SP], sTy[SR * SP];
  __shared__ T sce[CY * CX];
  const int n = c.n, cx = c.cx, P = c.P;  // n rows of cx cells
  const int ilo = blockIdx.x * TLX - H, jlo = blockIdx.y * TLY - H;
  const int I0 = (ilo >> 1) - 1, J0 = (jlo >> 1) - 1;
  if (xin && ec) {
    for (int p = threadIdx.x; p < CX * CY; p += NT) sce[p] = cd_at(ec, nc, cx / 2, Pc, I0 + p % CX, J0 + p / CX);
    __syncthreads();
  }
  for (int p = threadIdx.x; p < SR * SP; p += NT) {
    const int gi = ilo + p % SP, gj = jlo + p / SP;
    T vb = T(0), vx = T(0), vtx = T(0), vty = T(0);
    if (gi >= 0 && gj >= 0) {
      const long long gk = (long long)gj * P + gi;
      if (gi < cx && gj < n) {
        vb = b[gk];
        if (xin) {
          vx = xin[gk];
          if (ec) vx += prolong_D_sm(sce, CX, I0, J0, gi, gj);
        }
      }
      if (gi <= cx && gj < n) vtx = c.Tx[gk];
      if (gi < cx && gj <= n) vty = c.Ty[gk];
    }
    sb[p] = vb;
    sx0[p] = vx;
    sTx[p] = vtx;
    sTy[p] = vty;
  }
  __syncthreads();
  // shared view: global (i, j) -> (j - jlo) * SP + (i - ilo)
  const long long sh = (long long)jlo * SP + ilo;
  Coef<T> tc = c;
  tc.P = SP;
  tc.Tx = sTx - sh;
  tc.Ty = sTy - sh;
  const T* bq = sb - sh;
  T* dq = sd - sh;
  T* xa = sx0 - sh;
  T* xb = sx1 - sh;
  const T* cur = xin ? xa : nullptr;
  T* nxt = xb;
  // every point the first step computes is an interior cell: no boundary term anywhere
  const bool inner = ilo + 1 >= 1 && ilo + EX - 2 <= cx - 2 && jlo + 1 >= 1 && jlo + EY - 2 <= n - 2;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int lo = s + 1, w = EX - 2 * lo, hgt = EY - 2 * lo;
    if (inner) {
      for (int p = threadIdx.x; p < w * hgt; p += NT) {
        const int gi = ilo + lo + p % w, gj = jlo + lo + p / w;
        cheb_D_at<T, true>(tc, cur, bq, dq, nxt, cs.a[s], cs.c[s], gi, gj);
      }
    } else {
      for (int p = threadIdx.x; p < w * hgt; p += NT) {
        const int gi = ilo + lo + p % w, gj = jlo + lo + p / w;
        if (gi >= 0 && gj >= 0 && gi < cx && gj < n) cheb_D_at(tc, cur, bq, dq, nxt, cs.a[s], cs.c[s], gi, gj);
      }
    }
    __syncthreads();
    cur = nxt;
    nxt = (nxt == xb) ? xa : xb;
  }
  if constexpr (RR) {
    for (int p = threadIdx.x; p < TLX * TLY; p += NT) {
      const int gi = ilo + H + p % TLX, gj = jlo + H + p / TLX;
      if (gi >= cx || gj >= n) continue;
      const int k = gj * SP + gi;
      T off, dg;
      d_row(tc, cur, gi, gj, true, off, dg);
      dq[k] = bq[k] - (dg * cur[k] + off);
    }
    __syncthreads();
    const int I0 = (ilo + H) / 2, J0 = (jlo + H) / 2;
    for (int p = threadIdx.x; p < (TLX / 2) * (TLY / 2); p += NT) {
      const int I = I0 + p % (TLX / 2), J = J0 + p / (TLX / 2);
      if (I >= cx / 2 || J >= nc) continue;
      const T* r0 = dq + (2 * J) * SP + 2 * I;
      bco[(long long)J * Pc + I] = (r0[0] + r0[1]) + (r0[SP] + r0[SP + 1]);
    }
  }
  for (int p = threadIdx.x; p < TLX * TLY; p += NT) {
    const int gi = ilo + H + p % TLX, gj = jlo + H + p / TLX;
    if (gi < cx && gj < n) xout[(long long)gj * P + gi] = cur[(long long)gj * SP + gi];
  }
}

// RR (pre-smoothing from zero only): the tile also forms the residual b - A x
// of its output points and a ring of one around them (x is smoothed on a
// halo of NS + 2 for that) and restricts it to the coarse faces (I, J) whose
// fine face (2I, 2J) is one of its output points, into bco (nc x nc coarse
// cells, pitch Pc) -- the residual and restriction kernels of the level
// with their launches and the residual's round trip through memory, the same
// arithmetic per point.
template <typename T, int NS, int TLY, bool BT, bool RR = false, int NT = TLT>
__global__ void __launch_bounds__(NT, NT > TLT ? 2 : (TLY <= 8 ? 8 : 4))
    k_smooth_tile_V(Coef<T> c, const T* __restrict__ xin, const T* __restrict__ b, T* __restrict__ xout,
                    ChebSteps<T> cs, const T* __restrict__ ct, const T* __restrict__ ec, int nc, int Pc,
                    T* __restrict__ bco, Bat bt) {
  griddep_wait();
  // a separate instantiation for lockstep batches keeps the single-instance
  // kernel's coefficients in the parameter space
  if constexpr (BT) {
    long long o;
    if (!bat_enter(bt, o)) return;
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    xout = bsh(xout, o);
    ec = bsh(ec, o);
    bco = bsh(bco, o);
    if (ct) {
      const T* q = bsh(ct, o);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        cs.a[s] = q[s];
        cs.c[s] = q[8 + s];
      }
    }
  }
  constexpr int H = RR ? NS + 2 : NS, EX = TLX + 2 * H, EY = TLY + 2 * H, SP = EX + 1, SR = EY + 1;
  constexpr int CX = SP / 2 + 4, CY = SR / 2 + 4;  // coarse window of the prolongation
  __shared__ T sbu[SR * SP], sbv[SR * SP], sau[SR * SP], sav[SR * SP], sbu2[SR * SP], sbv2[SR * SP];
  __shared__ T sdu[SR * SP], sdv[SR * SP], sw[SP], srg[SP];
  __shared__ T scu[CY * CX], scv[CY * CX];
  const int n = c.n, nx = c.nx, P = c.P;
  const int nxc = nx / 2, iwc = c.iw / 2;  // the coarse level's width and interface window
  const long long nv = (long long)n * P;
  const int ilo = blockIdx.x * TLX - H, jlo = blockIdx.y * TLY - H;
  const T* ecu = ec;
  const T* ecv = ec ? ec + (long long)nc * Pc : nullptr;
  const int I0 = (ilo >> 1) - 1, J0 = (jlo >> 1) - 1;
  if (xin && ec) {
    // window entries no halo point reads are set to zero: coarse u faces
    // outside 0..nxc (which cu_at would read past its row on traction sides)
    // and coarse v rows below 0
    for (int p = threadIdx.x; p < CX * CY; p += NT) {
      const int I = I0 + p % CX, J = J0 + p / CX;
      scu[p] = (I >= 0 && I <= nxc) ? cu_at(ecu, nc, nxc, iwc, Pc, I, J, c.lat) : T(0);
      scv[p] = J >= 0 ? cv_at(ecv, nc, nxc, iwc, Pc, I, J) : T(0);
    }
    __syncthreads();
  }
  for (int p = threadIdx.x; p < SR * SP; p += NT) {
    const int gi = ilo + p % SP, gj = jlo + p / SP;
    T bu = T(0), bv = T(0), xu = T(0), xv = T(0);
    if (gi >= 0 && gj >= 0) {
      const long long gk = (long long)gj * P + gi;
      if (gi <= nx && gj < n) {  // u face
        bu = b[gk];
        if (xin) {
          xu = xin[gk];
          if (ec && (c.lat || (gi > 0 && gi < nx))) xu += prolong_u_sm(scu, CX, I0, J0, gi, gj);
        }
      }
      if (gi < nx && gj <= n) {  // v face (the Dirichlet ones take no increment)
        bv = b[nv + gk];
        if (xin) {
          xv = xin[nv + gk];
          if (ec && gj < n && (gj > 0 || on_gamma(c, gi))) xv += prolong_v_sm(scv, CX, I0, J0, gi, gj);
        }
      }
    }
    sbu[p] = bu;
    sbv[p] = bv;
    sau[p] = xu;
    sav[p] = xv;
  }
  for (int p = threadIdx.x; p < SP; p += NT) {
    const int gi = ilo + p;
    sw[p] = (gi >= 0 && gi <= nx) ? c.w[gi] : T(0);
    srg[p] = (gi >= 0 && gi < nx) ? c.rg[gi] : T(0);
  }
  __syncthreads();
  const long long sh = (long long)jlo * SP + ilo;
  Coef<T> tc = c;
  tc.P = SP;
  tc.w = sw - ilo;
  tc.rg = srg - ilo;
  const T* bu = sbu - sh;
  const T* bv = sbv - sh;
  T* du = sdu - sh;
  T* dv = sdv - sh;
  T* au = sau - sh;
  T* av = sav - sh;
  T* cu2 = sbu2 - sh;
  T* cv2 = sbv2 - sh;
  const T* curu = xin ? au : nullptr;
  const T* curv = xin ? av : nullptr;
  T* nxu = cu2;
  T* nxv = cv2;
  // every point the first step computes has interior u and v faces: no boundary term anywhere
  // (in the channel row 1 of the v faces reads the floor: interior from row 2)
  const bool inner = ilo + 1 >= 2 && ilo + EX - 2 <= nx - 2 && jlo + 1 >= (c.iw ? 2 : 1) && jlo + EY - 2 <= n - 2;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    const int lo = s + 1, w = EX - 2 * lo, hgt = EY - 2 * lo;
    if (inner) {
      for (int p = threadIdx.x; p < w * hgt; p += NT) {
        const int gi = ilo + lo + p % w, gj = jlo + lo + p / w;
        cheb_V_at2<T, true>(tc, curu, curv, bu, bv, du, dv, nxu, nxv, cs.a[s], cs.c[s], gi, gj);
      }
    } else {
      for (int p = threadIdx.x; p < w * hgt; p += NT) {
        const int gi = ilo + lo + p % w, gj = jlo + lo + p / w;
        if (gi >= 0 && gj >= 0 && gi <= nx && gj <= n)
          cheb_V_at2(tc, curu, curv, bu, bv, du, dv, nxu, nxv, cs.a[s], cs.c[s], gi, gj);
      }
    }
    __syncthreads();
    curu = nxu;
    curv = nxv;
    nxu = (nxu == cu2) ? au : cu2;
    nxv = (nxv == cv2) ? av : cv2;
  }
  if constexpr (RR) {
    // the residual (resid_V_at's arithmetic) into the d arrays, then the
    // coarse faces of the tile (restrict_V_at's arithmetic)
    constexpr int lo = NS + 1, w = EX - 2 * lo, hgt = EY - 2 * lo;
    for (int p = threadIdx.x; p < w * hgt; p += NT) {
      const int gi = ilo + lo + p % w, gj = jlo + lo + p / w;
      if (gi < 0 || gj < 0 || gi > nx || gj > n) continue;
      const int k = gj * SP + gi;
      if (gj < n) {
        T ax, dg = T(1);
        if ((gi == 0 || gi == nx) && !c.lat) {
          ax = curu[k];
        } else {
          T off;
          if (gi == 0 || gi == nx) ub_row(tc, curu, curv, gi, gj, true, off, dg);
          else u_row(tc, curu, curv, gi, gj, true, off, dg);
          ax = dg * curu[k] + off;
        }
        du[k] = bu[k] - ax;
      }
      if (gi < nx) {
        T ax, dg = T(1);
        if (gj == n || (gj == 0 && !on_gamma(c, gi))) {
          ax = curv[k];
        } else {
          T off;
          v_row(tc, curu, curv, gi, gj, true, off, dg);
          ax = dg * curv[k] + off;
        }
        dv[k] = bv[k] - ax;
      }
    }
    __syncthreads();
    const int I0 = (ilo + H) / 2, J0 = (jlo + H) / 2;
    for (int p = threadIdx.x; p < (TLX / 2) * (TLY / 2); p += NT) {
      const int I = I0 + p % (TLX / 2), J = J0 + p / (TLX / 2);
      if (I <= nxc && J <= nc) restrict_V_at2<T>(du, dv, SP, nc, nxc, iwc, Pc, bco, I, J, c.lat);
    }
  }
  for (int p = threadIdx.x; p < TLX * TLY; p += NT) {
    const int gi = ilo + H + p % TLX, gj = jlo + H + p / TLX;
    const long long gk = (long long)gj * P + gi, sk = (long long)gj * SP + gi;
    if (gi <= nx && gj < n) xout[gk] = curu[sk];
    if (gi < nx && gj <= n) xout[nv + gk] = curv[sk];
  }
}

// Launches with at most two tiles per SM in all (the GPU is otherwise idle
// there; a lockstep batch counts every instance's tiles) run 4-row tiles with
// 1024 threads instead of 256: a thread then takes a quarter of the points
// per step, which shortens the latency chain of the launch; every point's
// arithmetic is unchanged.
static const int TLT_SMALL = 1024;
static inline bool small_grid(const dim3& g) {
  if (t_conc) return false;  // other instances' launches share the GPU
  return (long long)g.x * g.y * (t_bat.off ? t_bat_n : 1) <= 2 * 152;
}

template <typename T, int NS, int TLY, bool RR>
void tile_D_go(const dim3& g, cudaStream_t s, const Coef<T>& c, const T* x_in, const T* b, T* x_out,
               const ChebSteps<T>& cs, const T* ct, const T* ec, int nc, int Pc, T* bco) {
  if constexpr (TLY == 4) {
    constexpr int NT = TLT_SMALL;
    if (small_grid(g)) {
      if (t_bat.off)
        launch_k(k_smooth_tile_D<T, NS, TLY, true, RR, NT>, g, dim3(NT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc,
                 Pc, bco);
      else
        launch_k(k_smooth_tile_D<T, NS, TLY, false, RR, NT>, g, dim3(NT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc,
                 Pc, bco);
      return;
    }
  }
  if (t_bat.off)
    launch_k(k_smooth_tile_D<T, NS, TLY, true, RR>, g, dim3(TLT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco);
  else launch_k(k_smooth_tile_D<T, NS, TLY, false, RR>, g, dim3(TLT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco);
}

template <typename T, int TLY, bool RR>
int launch_tile_D_rows(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct,
                       const T* ec, int nc, int Pc, T* bco, cudaStream_t s) {
  const dim3 g((c.cx + TLX - 1) / TLX, (c.n + TLY - 1) / TLY);
  switch (cs.ns) {
    case 1: tile_D_go<T, 1, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 2: tile_D_go<T, 2, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 3: tile_D_go<T, 3, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 4: tile_D_go<T, 4, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    default: return -1;
  }
  SD_COUNT(1);
  return 0;
}

template <typename T>
int launch_smooth_tile_D(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs,
                         const T* ct, const T* ec, int nc, int Pc, cudaStream_t s) {
  // (the register-column tiles take blocks of n x n cells: the Darcy block,
  // and the pressure Laplacian of the square geometry)
  if constexpr (std::is_same<T, float>::value)
    if (cs.wave && c.cx == c.n) return launch_wave_D(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s);
  if (cs.rows == 4) return launch_tile_D_rows<T, 4, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s);
  return cs.rows == 8 ? launch_tile_D_rows<T, 8, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s)
                      : launch_tile_D_rows<T, 16, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s);
}

template <typename T>
int launch_smooth_tile_D_rr(const Coef<T>& c, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct, int nc,
                            int Pc, T* bco, cudaStream_t s) {
  if (cs.wave || (c.n & 1)) return -1;
  if (cs.rows == 4) return launch_tile_D_rows<T, 4, true>(c, nullptr, b, x_out, cs, ct, nullptr, nc, Pc, bco, s);
  if (cs.rows == 8) return launch_tile_D_rows<T, 8, true>(c, nullptr, b, x_out, cs, ct, nullptr, nc, Pc, bco, s);
  return -1;
}

template <typename T, int NS, int TLY, bool RR>
void tile_V_go(const dim3& g, cudaStream_t s, const Coef<T>& c, const T* x_in, const T* b, T* x_out,
               const ChebSteps<T>& cs, const T* ct, const T* ec, int nc, int Pc, T* bco) {
  if constexpr (TLY == 4) {
    constexpr int NT = TLT_SMALL;
    if (small_grid(g)) {
      if (t_bat.off)
        launch_k(k_smooth_tile_V<T, NS, TLY, true, RR, NT>, g, dim3(NT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc,
                 Pc, bco);
      else
        launch_k(k_smooth_tile_V<T, NS, TLY, false, RR, NT>, g, dim3(NT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc,
                 Pc, bco);
      return;
    }
  }
  if (t_bat.off)
    launch_k(k_smooth_tile_V<T, NS, TLY, true, RR>, g, dim3(TLT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco);
  else launch_k(k_smooth_tile_V<T, NS, TLY, false, RR>, g, dim3(TLT), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco);
}

template <typename T, int TLY, bool RR>
int launch_tile_V_rows(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct,
                       const T* ec, int nc, int Pc, T* bco, cudaStream_t s) {
  const dim3 g((c.nx + 1 + TLX - 1) / TLX, (c.n + 1 + TLY - 1) / TLY);
  switch (cs.ns) {
    case 1: tile_V_go<T, 1, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 2: tile_V_go<T, 2, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 3: tile_V_go<T, 3, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    case 4: tile_V_go<T, 4, TLY, RR>(g, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc, bco); break;
    default: return -1;
  }
  SD_COUNT(1);
  return 0;
}

template <typename T>
int launch_smooth_tile_V(const Coef<T>& c, const T* x_in, const T* b, T* x_out, const ChebSteps<T>& cs,
                         const T* ct, const T* ec, int nc, int Pc, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value)
    if (cs.wave) return launch_wave_V(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s);
  if (cs.rows == 4) return launch_tile_V_rows<T, 4, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s);
  return cs.rows == 8 ? launch_tile_V_rows<T, 8, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s)
                      : launch_tile_V_rows<T, 16, false>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, nullptr, s);
}

template <typename T>
int launch_smooth_tile_V_rr(const Coef<T>& c, const T* b, T* x_out, const ChebSteps<T>& cs, const T* ct, int nc,
                            int Pc, T* bco, cudaStream_t s) {
  if (cs.wave || (c.n & 1)) return -1;
  if (cs.rows == 4) return launch_tile_V_rows<T, 4, true>(c, nullptr, b, x_out, cs, ct, nullptr, nc, Pc, bco, s);
  if (cs.rows == 8) return launch_tile_V_rows<T, 8, true>(c, nullptr, b, x_out, cs, ct, nullptr, nc, Pc, bco, s);
  return -1;
}

// ------------------------------------------------ fused coarse V-cycle
// All levels from `first` (at most 32 x 32 cells) down to the coarsest in one
// CTA: every work vector lives in shared memory (four per level: b, two
// iterates and d, which also holds the residual), the sweeps of the smoother,
// residual, transfers and the dense coarsest solve are separated by
// __syncthreads.  Same arithmetic, in the same order per point, as the
// per-level kernels; it only removes the launches of the small grids.  (Entry
// at 64 x 64 was measured slower than the per-level kernels it replaced.)
static __host__ __device__ inline int cyc_pitch(int n) { return ((n + 1) + 7) / 8 * 8; }
static __host__ __device__ inline int cyc_len(int n, int kind) {
  return kind == 0 ? (2 * n + 1) * cyc_pitch(n) : n * cyc_pitch(n);
}

// d = a d + c D^-1 (b - A x) at (i, j) of the velocity block (Dirichlet faces: d = 0)
template <typename T>
__device__ __forceinline__ void cheb_d_V_at(const Coef<T>& c, const T* __restrict__ x, const T* __restrict__ b,
                                            T* __restrict__ d, T a, T cc, int i, int j) {
  const int n = c.n, P = c.P;
  const T* u = x;
  const T* v = x + (long long)n * P;
  if (j < n) {
    const int k = j * P + i;
    if ((i == 0 || i == n) && !c.lat) {
      d[k] = T(0);
    } else {
      T off, dg;
      if (i == 0 || i == n) ub_row(c, u, v, i, j, true, off, dg);
      else u_row(c, u, v, i, j, true, off, dg);
      const T r = b[k] - (dg * x[k] + off);
      d[k] = (a != T(0) ? a * d[k] : T(0)) + sdiv(cc * r, dg);
    }
  }
  if (i < n) {
    const int k = n * P + j * P + i;
    if (j == n) {
      d[k] = T(0);
    } else {
      T off, dg;
      v_row(c, u, v, i, j, true, off, dg);
      const T r = b[k] - (dg * x[k] + off);
      d[k] = (a != T(0) ? a * d[k] : T(0)) + sdiv(cc * r, dg);
    }
  }
}

template <typename T>
__device__ __forceinline__ void cheb_d_D_at(const Coef<T>& c, const T* __restrict__ x, const T* __restrict__ b,
                                            T* __restrict__ d, T a, T cc, int i, int j) {
  const int k = j * c.P + i;
  T off, dg;
  d_row(c, x, i, j, true, off, dg);
  const T r = b[k] - (dg * x[k] + off);
  d[k] = (a != T(0) ? a * d[k] : T(0)) + sdiv(cc * r, dg);
}

// ops: 0 Chebyshev step (writes d and x_out from x_in), 1 d-update only,
//      2 x += d, 3 residual into d, 4 restriction of d to level l + 1,
//      5 prolongation of level l + 1 into x
template <typename T>
__device__ void cyc_sweep(const CoarseCycle<T>& q, int l, int op, T* X, const T* B, T* D, T a, T cc, T* Bc,
                          const T* Xc) {
  const Coef<T>& c = q.c[l];
  const int n = c.n;
  const int w = q.kind == 0 ? n + 1 : n;
  const int nc = (op >= 4) ? q.c[l + 1].n : 0;
  const int wc = q.kind == 0 ? nc + 1 : nc;
  const int npts = op == 4 ? wc * wc : w * w;
  for (int p = threadIdx.x; p < npts; p += blockDim.x) {
    const int ww = op == 4 ? wc : w;
    const int i = p % ww, j = p / ww;
    if (op == 0) {  // Chebyshev step x_out (X) = x_in (Xc, null: zero) + d
      if (q.kind == 0) cheb_V_at(c, Xc, B, D, X, a, cc, i, j);
      else cheb_D_at(c, Xc, B, D, X, a, cc, i, j);
    } else if (op == 1) {
      if (q.kind == 0) cheb_d_V_at(c, X, B, D, a, cc, i, j);
      else cheb_d_D_at(c, X, B, D, a, cc, i, j);
    } else if (op == 2) {
      if (q.kind == 0) {
        if (j < n) X[j * c.P + i] += D[j * c.P + i];
        if (i < n) X[(n + j) * c.P + i] += D[(n + j) * c.P + i];
      } else {
        X[j * c.P + i] += D[j * c.P + i];
      }
    } else if (op == 3) {
      if (q.kind == 0) resid_V_at(c, X, B, D, 0, i, j);
      else resid_D_at(c, X, B, D, 0, i, j);
    } else if (op == 4) {
      if (q.kind == 0) restrict_V_at(n, c.P, D, nc, nc, 0, q.c[l + 1].P, Bc, i, j, c.lat);
      else restrict_D_at(c.P, D, q.c[l + 1].P, Bc, i, j);
    } else {
      if (q.kind == 0) prolong_V_at(n, c.P, X, nc, nc, 0, q.c[l + 1].P, Xc, i, j, c.lat);
      else prolong_D_at(c.P, X, nc, nc, q.c[l + 1].P, Xc, i, j);
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void coarse_cycle_body(const CoarseCycle<T>& q) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  T* B[SD_CYC_MAXL];
  T* X[SD_CYC_MAXL];
  T* X2[SD_CYC_MAXL];
  T* D[SD_CYC_MAXL];
  T* cur[SD_CYC_MAXL];
  int off = 0;
  for (int l = 0; l < q.nlev; ++l) {
    const int len = cyc_len(q.c[l].n, q.kind);
    B[l] = sm + off; off += len;
    X[l] = sm + off; off += len;
    X2[l] = sm + off; off += len;
    D[l] = sm + off; off += len;
  }
  const int len0 = cyc_len(q.c[0].n, q.kind);
  for (int p = threadIdx.x; p < len0; p += blockDim.x) B[0][p] = q.b_in[p];
  __syncthreads();
  const int L = q.nlev;
  for (int l = 0; l + 1 < L; ++l) {
    T* c0 = nullptr;
    for (int k = 0; k < q.deg[l]; ++k) {
      T* o = (c0 == X[l]) ? X2[l] : X[l];
      cyc_sweep<T>(q, l, 0, o, B[l], D[l], q.cha[l][k], q.chc[l][k], nullptr, c0);
      c0 = o;
    }
    cur[l] = c0;
    cyc_sweep<T>(q, l, 3, c0, B[l], D[l], T(0), T(0), nullptr, nullptr);
    cyc_sweep<T>(q, l, 4, c0, B[l], D[l], T(0), T(0), B[l + 1], nullptr);
  }
  {  // coarsest grid: x = A^-1 b with the FP64 inverse
    const int m = q.m;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int r = warp; r < m; r += nw) {
      const double* row = q.Ainv + (long long)r * m;
      double s = 0.0;
      for (int l2 = lane; l2 < m; l2 += 32) s = fma(row[l2], (double)B[L - 1][q.idx[l2]], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
      if (lane == 0) X[L - 1][q.idx[r]] = (T)s;
    }
    cur[L - 1] = X[L - 1];
    __syncthreads();
  }
  for (int l = L - 2; l >= 0; --l) {
    cyc_sweep<T>(q, l, 5, cur[l], B[l], D[l], T(0), T(0), nullptr, cur[l + 1]);
    T* c0 = cur[l];
    for (int k = 0; k < q.deg[l]; ++k) {
      T* o = (c0 == X[l]) ? X2[l] : X[l];
      cyc_sweep<T>(q, l, 0, o, B[l], D[l], q.cha[l][k], q.chc[l][k], nullptr, c0);
      c0 = o;
    }
    cur[l] = c0;
  }
  // write the valid entries of the first level's result
  const Coef<T>& c = q.c[0];
  const int n = c.n, w = q.kind == 0 ? n + 1 : n;
  for (int p = threadIdx.x; p < w * w; p += blockDim.x) {
    const int i = p % w, j = p / w;
    if (q.kind == 0) {
      if (j < n) q.x_out[(long long)j * c.P + i] = cur[0][j * c.P + i];
      if (i < n) q.x_out[(long long)(n + j) * c.P + i] = cur[0][(n + j) * c.P + i];
    } else {
      q.x_out[(long long)j * c.P + i] = cur[0][j * c.P + i];
    }
  }
}

// The descriptor is copied to shared memory first; in a lockstep batch it is
// then moved to this block's instance (its arrays by the instance offset,
// its Chebyshev coefficients read from the instance's own table).  A single
// instance runs the same code on the unmoved copy, so both compile to the
// same arithmetic and give bitwise the same result.
template <typename T>
__global__ void __launch_bounds__(1024) k_coarse_cycle(const __grid_constant__ CoarseCycle<T> q, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  __shared__ CoarseCycle<T> sq;
  {
    const int* src = reinterpret_cast<const int*>(&q);
    int* dst = reinterpret_cast<int*>(&sq);
    for (int w = threadIdx.x; w < (int)(sizeof(CoarseCycle<T>) / sizeof(int)); w += blockDim.x) dst[w] = src[w];
  }
  __syncthreads();
  if (bt.off) {  // uniform over the block
    const int tid = threadIdx.x;
    if (tid < q.nlev) bsh_coef(sq.c[tid], o);
    if (tid >= 32 && tid < 32 + 8 * q.nlev) {
      const int l = (tid - 32) >> 3, k = (tid - 32) & 7;
      if (q.cht[l] && k < q.deg[l]) {
        const T* row = bsh(q.cht[l], o);
        sq.cha[l][k] = row[k];
        sq.chc[l][k] = row[8 + k];
      }
    }
    if (tid == 96) {
      sq.Ainv = bsh(q.Ainv, o);
      sq.idx = bsh(q.idx, o);
      sq.b_in = bsh(q.b_in, o);
      sq.x_out = bsh(q.x_out, o);
    }
    __syncthreads();
  }
  coarse_cycle_body(sq);
}

template <typename T>
size_t coarse_cycle_smem(const CoarseCycle<T>& q) {
  size_t tot = 0;
  for (int l = 0; l < q.nlev; ++l) tot += 4 * (size_t)cyc_len(q.c[l].n, q.kind);
  return tot * sizeof(T);
}

template <typename T>
int prepare_coarse_cycle() {
  return cudaFuncSetAttribute(k_coarse_cycle<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) ==
                 cudaSuccess
             ? 0
             : -1;
}

template <typename T>
int launch_coarse_cycle(const CoarseCycle<T>& q, cudaStream_t s) {
  const size_t sm = coarse_cycle_smem(q);
  if (sm > 200 * 1024) return -1;
  SD_COUNT(1);
  launch_k(k_coarse_cycle<T>, dim3(1), dim3(1024), sm, s, q);
  return 0;
}

// ------------------------------------------------------ preconditioner glue
// Block upper-triangular Stokes part (Sec. 4, zero block replaced by the
// Schur approximation S^ = h^2/(2 mu) I, or by I): z_pf = schur * r_pf,
// then the velocity rhs r_v - B z_pf for the V-block multigrid.
// rs (may be null: 1) in these glue kernels: the scale of r, the Krylov
// basis vector kept unnormalised (r is used as rs[0] r, formed in FP64 before
// the conversion, so the multigrid sees the same values as from a normalised
// vector).
template <typename T>
__global__ void k_precond_entry(Coef<double> c, const double* __restrict__ r, double* __restrict__ z, T schur,
                                const T* __restrict__ eP, T cmass, T hT, int useB, int useB1, T* __restrict__ rV,
                                const double* __restrict__ rs, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    r = bsh(r, o);
    z = bsh(z, o);
    eP = bsh(eP, o);
    rV = bsh(rV, o);
    rs = bsh(rs, o);
  }
  const double sr = rs ? rs[0] : 1.0;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n, nx = c.nx, P = c.P;
  const T h = hT;  // parameters arrive in T: an FP64 conversion per thread would run on the FP64 pipe
  const double* rpf = r + (long long)(2 * n + 1) * P;
  // z_pf at cell kc: schur * r_pf (+ cmass * eP, the pressure-Laplacian part),
  // evaluated in the multigrid precision T, once per cell of the block and its
  // west and south neighbours (staged in shared memory: each FP64 value is
  // converted once)
  const T ts = schur, tm = cmass;
  auto zp = [&](long long kc) -> T { return ts * (T)(rpf[kc] * sr) + (eP ? tm * eP[kc] : T(0)); };
  __shared__ T sz[BY + 1][BX + 1];
  const int i0 = blockIdx.x * blockDim.x - 1, j0 = blockIdx.y * blockDim.y - 1;
  for (int p = threadIdx.y * blockDim.x + threadIdx.x; p < (BX + 1) * (BY + 1); p += BX * BY) {
    const int ci = i0 + p % (BX + 1), cj = j0 + p / (BX + 1);
    sz[p / (BX + 1)][p % (BX + 1)] = (ci >= 0 && ci < nx && cj >= 0 && cj < n) ? zp((long long)cj * P + ci) : T(0);
  }
  __syncthreads();
  if (i > nx || j > n) return;
  const int li = threadIdx.x + 1, lj = threadIdx.y + 1;
  const T zc = sz[lj][li];
  if (i < nx && j < n) z[(long long)(2 * n + 1) * P + (long long)j * P + i] = (double)zc;
  if (j < n) {
    const long long k = (long long)j * P + i;
    T val = (T)(r[k] * sr);
    if (useB && i > 0 && i < nx) val -= h * (zc - sz[lj][li - 1]);
    else if (useB && c.lat) val -= i == 0 ? h * zc : -h * sz[lj][li - 1];  // traction side
    rV[k] = val;
  }
  if (i < nx) {
    const long long kv = (long long)j * P + i;
    const long long k = (long long)n * P + kv;
    T val = (T)(r[k] * sr);
    const bool iface = j == 0 && on_gamma(c, i);  // (a floor face beside it is a Dirichlet row)
    if (useB && j < n && (j > 0 || iface)) {
      if (j > 0) val -= h * (zc - sz[lj - 1][li]);
      else val -= h * zc;
    }
    // Darcy solved first: r_v - B'_1 z_pm on the interface rows (B'_1 = -h)
    if (useB1 && iface) val += h * (T)z[(long long)(3 * n + 1) * P + (long long)(n - 1) * P + i - c.iw];
    rV[k] = val;
  }
}

template <typename T>
void launch_precond_entry(const Coef<double>& c, const double* r, double* z, double schur, const T* eP, double cmass,
                          int use_B, int use_B1, T* rV, cudaStream_t s, const double* rs) {
  SD_COUNT(1);
  launch_k(k_precond_entry<T>, dim3(grid2(c.nx + 1, c.n + 1)), dim3(dim3(BX, BY)), 0, s, c, r, z, (T)schur, eP,
           (T)cmass, (T)c.h, use_B, use_B1, rV, rs);
}

template <typename T>
__global__ void k_precond_mid(Coef<double> c, const double* __restrict__ r, double* __restrict__ z,
                              const T* __restrict__ eV, int useC, T* __restrict__ rD, const double* __restrict__ rs,
                              Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    r = bsh(r, o);
    z = bsh(z, o);
    eV = bsh(eV, o);
    rD = bsh(rD, o);
    rs = bsh(rs, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n, P = c.P;
  if (i > c.nx || j > n) return;
  if (j < n) {
    const long long k = (long long)j * P + i;
    z[k] = (double)eV[k];
  }
  if (i < c.nx) {
    const long long k = (long long)n * P + (long long)j * P + i;
    z[k] = (double)eV[k];
  }
  if (rD && i < n && j < n) {
    const long long kc = (long long)j * P + i;
    T val = (T)(r[(long long)(3 * n + 1) * P + kc] * (rs ? rs[0] : 1.0));
    if (useC && j == n - 1) val -= (T)c.h * eV[(long long)n * P + c.iw + i];
    rD[kc] = val;
  }
}

template <typename T>
void launch_precond_mid(const Coef<double>& c, const double* r, double* z, const T* eV, int use_C, T* rD,
                        cudaStream_t s, const double* rs) {
  SD_COUNT(1);
  launch_k(k_precond_mid<T>, dim3(grid2(c.nx + 1, c.n + 1)), dim3(dim3(BX, BY)), 0, s, c, r, z, eV, use_C, rD, rs);
}

template <typename T>
__global__ void k_precond_exit(int n, int P, double* __restrict__ z, const T* __restrict__ eD, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    z = bsh(z, o);
    eD = bsh(eD, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  const long long kc = (long long)j * P + i;
  z[(long long)(3 * n + 1) * P + kc] = (double)eD[kc];
}

template <typename T>
void launch_precond_exit(const Coef<double>& c, double* z, const T* eD, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_precond_exit<T>, dim3(grid2(c.n, c.n)), dim3(dim3(BX, BY)), 0, s, c.n, c.P, z, eD);
}

// P^pv_BGS(P_V, P_D') of Sec. 4: after z_v = P_V r_v, the identity block
// gives z_pf = r_pf - C z_v (C: the continuity rows of Eq. (2)).
template <typename T>
__global__ void k_precond_bgs_pff(Coef<double> c, const double* __restrict__ r, double* __restrict__ z,
                                  const T* __restrict__ eV, const double* __restrict__ rs, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    bsh_coef(c, o);
    r = bsh(r, o);
    z = bsh(z, o);
    eV = bsh(eV, o);
    rs = bsh(rs, o);
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n, P = c.P;
  if (i >= c.nx || j >= n) return;
  const long long kc = (long long)j * P + i;
  const T* u = eV;
  const T* v = eV + (long long)n * P;
  double s = (j > 0 || on_gamma(c, i)) ? -(double)v[kc] : 0.0;
  if (c.lat || i + 1 <= c.nx - 1) s += (double)u[kc + 1];
  if (c.lat || i >= 1) s -= (double)u[kc];
  if (j + 1 <= n - 1) s += (double)v[kc + P];
  const long long kp = (long long)(2 * n + 1) * P + kc;
  z[kp] = r[kp] * (rs ? rs[0] : 1.0) - c.h * s;
}

template <typename T>
void launch_precond_bgs_pff(const Coef<double>& c, const double* r, double* z, const T* eV, cudaStream_t s,
                            const double* rs) {
  SD_COUNT(1);
  launch_k(k_precond_bgs_pff<T>, dim3(grid2(c.nx, c.n)), dim3(dim3(BX, BY)), 0, s, c, r, z, eV, rs);
}

// ------------------------------------------------------------------ setup
__global__ void k_pack_K(const double* __restrict__ Kd, int n, double* __restrict__ Kp, int P) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= n || j >= n) return;
  Kp[(long long)j * P + i] = Kd[(long long)j * n + i];
}
void launch_pack_K(const double* Kdense, int n, double* Kp, int P, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_pack_K, dim3(grid2(n, n)), dim3(dim3(BX, BY)), 0, s, Kdense, n, Kp, P);
}

__global__ void k_fill_K(double* __restrict__ K, int cx, int n, int P, double v) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= cx || j >= n) return;
  K[(long long)j * P + i] = v;
}
void launch_fill_K(double* K, int cx, int n, int P, double v, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_fill_K, dim3(grid2(cx, n)), dim3(dim3(BX, BY)), 0, s, K, cx, n, P, v);
}

// coarse permeability: geometric mean of the 2 x 2 children
__global__ void k_coarsen_K(const double* __restrict__ Kf, int nf, int Pf, double* __restrict__ Kc, int Pc) {
  griddep_wait();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nc = nf / 2;
  if (I >= nc || J >= nc) return;
  const double* k0 = Kf + (long long)(2 * J) * Pf + 2 * I;
  Kc[(long long)J * Pc + I] = sqrt(sqrt(k0[0] * k0[1] * k0[Pf] * k0[Pf + 1]));
}
void launch_coarsen_K(const double* Kf, int nf, int Pf, double* Kc, int Pc, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_coarsen_K, dim3(grid2(nf / 2, nf / 2)), dim3(dim3(BX, BY)), 0, s, Kf, nf, Pf, Kc, Pc);
}

// One coefficient set over cx x n cells of K (Tx, Ty) and the interface
// coefficients of the free-flow floor (w, rg).  lat: traction free-flow sides
// (BJS coefficients of the square's interface corners); xdir: the x boundary
// faces are Dirichlet over the half cell (2K/mu) instead of no-flow -- the
// pressure Laplacian of the Schur block with traction sides, where the side u
// faces, like v_Gamma, have half-volume mass; [b0, b1): the cells whose
// bottom face is Dirichlet (2K/mu), the others no-flow.  w over u faces
// 0..nx and rg over floor faces 0..nx-1 read the top row of K, which lies
// under floor faces iw .. iw + n - 1 (the channel's interface ends take the
// one pm cell beside them).
template <typename T>
__global__ void k_setup_coef(const double* __restrict__ K, int n, int cx, int P, double mu, double alpha, int lat,
                             int xdir, int b0, int b1, int nx, int iw, T* w, T* rg, T* Tx, T* Ty) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (j > n) return;
  const double h = 1.0 / n;
  if (j < n && i <= cx) {  // x faces of row j
    double t = 0.0;
    if (i > 0 && i < cx) {
      const double ka = K[(long long)j * P + i - 1], kb = K[(long long)j * P + i];
      t = 2.0 * ka * kb / (ka + kb) / mu;
    } else if (xdir) {
      t = 2.0 * K[(long long)j * P + (i == 0 ? 0 : cx - 1)] / mu;
    }
    Tx[(long long)j * P + i] = (T)t;
  }
  if (i < cx) {  // y faces below row j
    double t = 0.0;
    if (j == 0) {
      if (i >= b0 && i < b1) t = 2.0 * K[i] / mu;
    } else if (j < n) {
      const double ka = K[(long long)(j - 1) * P + i], kb = K[(long long)j * P + i];
      t = 2.0 * ka * kb / (ka + kb) / mu;
    }
    Ty[(long long)j * P + i] = (T)t;
  }
  if (j == 0 && i <= nx) {
    const double* top = K + (long long)(n - 1) * P;
    const int p = i - iw;
    if (p > 0 && p < n) {
      const double beta = 0.5 * (sqrt(top[p - 1]) + sqrt(top[p])) / alpha;
      w[i] = (T)(mu / (h + 2.0 * beta));
    } else if ((p == 0 || p == n) && (lat || iw > 0)) {  // an end of the interface: the one pm cell below
      const double beta = sqrt(top[p == 0 ? 0 : n - 1]) / alpha;
      w[i] = (T)(mu / (h + 2.0 * beta));
    } else {
      w[i] = (T)0;
    }
    if (i < nx) rg[i] = (p >= 0 && p < n) ? (T)(mu * h * h / (2.0 * top[p])) : (T)0;
  }
}

template <typename T>
void launch_setup_coef(const double* Kp, int n, int cx, int P, double mu, double alpha, int lat, int xdir, int b0,
                       int b1, int nx, int iw, T* w, T* rg, T* Tx, T* Ty, cudaStream_t s) {
  SD_COUNT(1);
  const int wx = (cx > nx ? cx : nx) + 1;
  launch_k(k_setup_coef<T>, dim3(grid2(wx, n + 1)), dim3(dim3(BX, BY)), 0, s, Kp, n, cx, P, mu, alpha, lat, xdir, b0,
           b1, nx, iw, w, rg, Tx, Ty);
}

// The Darcy rows of the cells below Gamma carry + h v_Gamma (C'_1) and the
// v_Gamma rows - h p_pm (B'_1); eliminating v_Gamma with the diagonal d of its
// row adds h^2 / d to those Darcy rows' diagonal.  In the cell rows a top-face
// coefficient enters the diagonal alone (the face above row n - 1 has no
// neighbour), so the correction is stored as that coefficient.  d is the
// v_Gamma row's diagonal as the velocity block forms it.
__global__ void k_darcy_schur_top(double* __restrict__ TyR, const double* __restrict__ w,
                                  const double* __restrict__ rg, int n, int nx, int iw, int P, double mu, double cm,
                                  double h, int lat) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int f = iw + i;
  const bool left = f == 0, right = f == nx - 1;
  const double wl = (left && !lat) ? 0.0 : w[f], wr = (right && !lat) ? 0.0 : w[f + 1];
  double d = 0.5 * cm + 2.0 * mu + rg[f];
  d += left ? (lat ? h * wl : mu) : 0.5 * h * wl;
  d += right ? (lat ? h * wr : mu) : 0.5 * h * wr;
  TyR[(long long)n * P + i] = h * h / d;
}

void launch_darcy_schur_top(double* TyR, const double* w, const double* rg, int n, int nx, int iw, int P, double mu,
                            double cm, double h, int lat, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_darcy_schur_top, dim3((n + 127) / 128), dim3(128), 0, s, TyR, w, rg, n, nx, iw, P, mu, cm, h, lat);
}

template <typename T>
__global__ void k_convert(const double* __restrict__ a, T* __restrict__ b, long long len,
                          const double* __restrict__ rs, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    a = bsh(a, o);
    b = bsh(b, o);
    rs = bsh(rs, o);
  }
  const double sr = rs ? rs[0] : 1.0;  // the scale of a (as in the glue kernels)
  // 32-bit indices (a vector has fewer than 2^31 entries); the conversion
  // itself runs on the FP64 pipe
  const int n = (int)len;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) b[k] = (T)(a[k] * sr);
}
template <typename T>
void launch_convert(const double* src, T* dst, long long len, cudaStream_t s, const double* rs) {
  SD_COUNT(1);
  long long nb = (len + 255) / 256;
  if (nb > 4096) nb = 4096;
  if (nb < 1) nb = 1;
  launch_k(k_convert<T>, dim3((int)nb), dim3(256), 0, s, src, dst, len, rs);
}

// ------------------------------------------------- manufactured solution
// psi = sin(pi x) phi(y), phi = 1 + A(y-1) + (y-1)^2, A = pi^2 + 2;
// u = psi_y, v = -psi_x, p_ff = cos(pi x)(1 - 2 mu pi A), p_pm = cos(pi x) e^{pi(y-1)},
// every field times s = 1 + t.  The momentum source f = dv/dt - mu lap v + grad p
// splits as f = f0 + s f1 with f0 = (U0, V0) (the time derivative) and
// f1 = (mu pi^2 U0 - pi c0 sin(pi x), -mu pi cos(pi x)(pi^2 phi - 2)).
#define SD_PI 3.14159265358979323846
__device__ __forceinline__ double mm_A() { return SD_PI * SD_PI + 2.0; }
__device__ __forceinline__ double mm_phi(double y) { const double s = y - 1.0; return 1.0 + mm_A() * s + s * s; }
__device__ __forceinline__ double mm_U0(double x, double y) { return sin(SD_PI * x) * (mm_A() + 2.0 * (y - 1.0)); }
__device__ __forceinline__ double mm_V0(double x, double y) { return -SD_PI * cos(SD_PI * x) * mm_phi(y); }
__device__ __forceinline__ double mm_Pff0(double x, double mu) { return cos(SD_PI * x) * (1.0 - 2.0 * mu * SD_PI * mm_A()); }
__device__ __forceinline__ double mm_Ppm0(double x, double y) { return cos(SD_PI * x) * exp(SD_PI * (y - 1.0)); }
__device__ __forceinline__ double mm_f1x(double x, double y, double mu) {
  return mu * SD_PI * SD_PI * mm_U0(x, y) - SD_PI * (1.0 - 2.0 * mu * SD_PI * mm_A()) * sin(SD_PI * x);
}
__device__ __forceinline__ double mm_f1y(double x, double y, double mu) {
  return -mu * SD_PI * cos(SD_PI * x) * (SD_PI * SD_PI * mm_phi(y) - 2.0);
}

// B0: time-derivative part of the integrated source; B1: all terms proportional
// to the time function s1 (1 + t for the manufactured cases: the rest of the
// source, boundary data moved to the right-hand side, Dirichlet values of the
// identity rows; p_in(t) for the pressure-driven problem: the inflow traction).
//   bc 0: Dirichlet free-flow sides; bc 1: traction sides with the
//   manufactured data (P_b = p - 2 mu du/dx, V_b = v on x = 0, 1);
//   bc 2: the pressure-driven problem (unit inflow traction on the left
//   side, all other data and sources zero).
__device__ __forceinline__ double mm_Pside(double x, double y, double mu) {  // p - 2 mu du/dx at s = 1
  return mm_Pff0(x, mu) - 2.0 * mu * SD_PI * cos(SD_PI * x) * (mm_A() + 2.0 * (y - 1.0));
}

__global__ void k_mms_terms(Coef<double> c, int bc, const double* __restrict__ K, double* __restrict__ B0,
                            double* __restrict__ B1) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n, P = c.P;
  if (i > n || j > n) return;
  const double h = c.h, mu = c.mu, h2 = h * h;
  const bool lat = bc != 0, mms = bc != 2;
  if (j < n) {  // u face (i, j)
    const long long k = (long long)j * P + i;
    const double x = i * h, y = 1.0 + (j + 0.5) * h;
    double b0 = 0.0, b1 = 0.0;
    if ((i == 0 || i == n) && !lat) {
      b1 = mm_U0(x, y);
    } else if (i == 0 || i == n) {  // traction side, half control volume
      const double sg = i == 0 ? 1.0 : -1.0;
      if (mms) {
        b0 = 0.5 * h2 * mm_U0(x, y);
        b1 = 0.5 * h2 * mm_f1x(x, y, mu) + sg * h * mm_Pside(x, y, mu);
        if (j < n - 1) b1 -= sg * mu * mm_V0(x, 1.0 + (j + 1) * h);
        else b1 += mu * mm_U0(x, 2.0) + sg * mu * (mm_V0(x + sg * 0.5 * h, 2.0) - mm_V0(x, 2.0));
        if (j > 0) b1 += sg * mu * mm_V0(x, 1.0 + j * h);
        else b1 += sg * h * c.w[i] * mm_V0(x, 1.0);
      } else if (i == 0) {
        b1 = h;  // inflow traction p_in(t) enters as s1
      }
    } else if (mms) {
      b0 = h2 * mm_U0(x, y);
      b1 = h2 * mm_f1x(x, y, mu);
      if (i == 1 && !lat) b1 += 2.0 * mu * mm_U0(0.0, y);
      if (i == n - 1 && !lat) b1 += 2.0 * mu * mm_U0(1.0, y);
      if (j == n - 1) b1 += 2.0 * mu * mm_U0(x, 2.0) + mu * (mm_V0(x + 0.5 * h, 2.0) - mm_V0(x - 0.5 * h, 2.0));
    }
    B0[k] = b0;
    B1[k] = b1;
  }
  if (i < n) {  // v face (i, j)
    const long long k = (long long)n * P + (long long)j * P + i;
    const double x = (i + 0.5) * h, y = 1.0 + j * h;
    double b0 = 0.0, b1 = 0.0;
    if (!mms) {
    } else if (j == n) {
      b1 = mm_V0(x, 2.0);
    } else if (j == 0) {
      b0 = 0.5 * h2 * mm_V0(x, 1.0);
      b1 = 0.5 * h2 * mm_f1y(x, 1.0, mu);
      if (i == 0) {
        if (lat) b1 += h * c.w[0] * mm_V0(0.0, 1.0);
        else b1 += -mu * (mm_U0(0.0, 1.0 + 0.5 * h) - mm_U0(0.0, 1.0)) + mu * mm_V0(0.0, 1.0);
      }
      if (i == n - 1) {
        if (lat) b1 += h * c.w[n] * mm_V0(1.0, 1.0);
        else b1 += mu * (mm_U0(1.0, 1.0 + 0.5 * h) - mm_U0(1.0, 1.0)) + mu * mm_V0(1.0, 1.0);
      }
    } else {
      b0 = h2 * mm_V0(x, y);
      b1 = h2 * mm_f1y(x, y, mu);
      if (j == n - 1) b1 += 2.0 * mu * mm_V0(x, 2.0);
      if (i == 0) {
        if (lat) b1 += 2.0 * mu * mm_V0(0.0, y);
        else b1 += 2.0 * mu * mm_V0(0.0, y) - mu * (mm_U0(0.0, y + 0.5 * h) - mm_U0(0.0, y - 0.5 * h));
      }
      if (i == n - 1) {
        if (lat) b1 += 2.0 * mu * mm_V0(1.0, y);
        else b1 += 2.0 * mu * mm_V0(1.0, y) + mu * (mm_U0(1.0, y + 0.5 * h) - mm_U0(1.0, y - 0.5 * h));
      }
    }
    B0[k] = b0;
    B1[k] = b1;
  }
  if (i < n && j < n) {
    const long long kc = (long long)j * P + i;
    const double y = 1.0 + (j + 0.5) * h, x = (i + 0.5) * h;
    double s = 0.0;
    if (mms) {
      if (i == 0 && !lat) s += h * mm_U0(0.0, y);
      if (i == n - 1 && !lat) s -= h * mm_U0(1.0, y);
      if (j == n - 1) s -= h * mm_V0(x, 2.0);
    }
    B0[(long long)(2 * n + 1) * P + kc] = 0.0;
    B1[(long long)(2 * n + 1) * P + kc] = s;
    double sp = 0.0;
    if (j == 0 && mms) sp = 2.0 * K[i] / mu * mm_Ppm0(x, 0.0);
    B0[(long long)(3 * n + 1) * P + kc] = 0.0;
    B1[(long long)(3 * n + 1) * P + kc] = sp;
  }
}

// The same terms for the channel (free flow x in [-1, 2], c.nx = 3n cells
// across, the interface under floor faces c.iw .. c.iw + n - 1): the
// manufactured solution is the same expression continued in x.  What the
// floor beside the interface adds: its v faces are Dirichlet rows (value v at
// y = 1); the u faces above it see the wall at half distance (u and the
// tangential derivative of v there are data); at the two ends of the
// interface the wall face beside the eliminated slip, and beside the half
// control volume of v_Gamma, enters as data; the v faces of row 1 and the
// continuity rows of row 0 above the wall take the wall face's value.  The
// traction ends x = -1, 2 meet the floor wall at half distance.
__global__ void k_mms_terms_ch(Coef<double> c, int bc, const double* __restrict__ K, double* __restrict__ B0,
                               double* __restrict__ B1) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = c.n, nx = c.nx, iw = c.iw, P = c.P;
  if (i > nx || j > n) return;
  const double h = c.h, mu = c.mu, h2 = h * h;
  const double xl = -1.0, xr = 2.0;
  const bool lat = bc != 0, mms = bc != 2;
  if (j < n) {  // u face (i, j)
    const long long k = (long long)j * P + i;
    const double x = (i - iw) * h, y = 1.0 + (j + 0.5) * h;
    double b0 = 0.0, b1 = 0.0;
    if ((i == 0 || i == nx) && !lat) {
      b1 = mm_U0(x, y);
    } else if (i == 0 || i == nx) {  // traction end, half control volume
      const double sg = i == 0 ? 1.0 : -1.0;
      if (mms) {
        b0 = 0.5 * h2 * mm_U0(x, y);
        b1 = 0.5 * h2 * mm_f1x(x, y, mu) + sg * h * mm_Pside(x, y, mu);
        if (j < n - 1) b1 -= sg * mu * mm_V0(x, 1.0 + (j + 1) * h);
        else b1 += mu * mm_U0(x, 2.0) + sg * mu * (mm_V0(x + sg * 0.5 * h, 2.0) - mm_V0(x, 2.0));
        if (j > 0) b1 += sg * mu * mm_V0(x, 1.0 + j * h);
        else b1 += mu * mm_U0(x, 1.0) - sg * mu * (mm_V0(x + sg * 0.5 * h, 1.0) - mm_V0(x, 1.0));
      } else if (i == 0) {
        b1 = h;  // inflow traction p_in(t) enters as s1
      }
    } else if (mms) {
      b0 = h2 * mm_U0(x, y);
      b1 = h2 * mm_f1x(x, y, mu);
      if (i == 1 && !lat) b1 += 2.0 * mu * mm_U0(xl, y);
      if (i == nx - 1 && !lat) b1 += 2.0 * mu * mm_U0(xr, y);
      if (j == n - 1) b1 += 2.0 * mu * mm_U0(x, 2.0) + mu * (mm_V0(x + 0.5 * h, 2.0) - mm_V0(x - 0.5 * h, 2.0));
      if (j == 0) {
        if (i >= iw && i <= iw + n) {
          const double wh = c.w[i] * h;
          if (!on_gamma(c, i)) b1 -= wh * mm_V0(x + 0.5 * h, 1.0);
          if (!on_gamma(c, i - 1)) b1 += wh * mm_V0(x - 0.5 * h, 1.0);
        } else {
          b1 += 2.0 * mu * mm_U0(x, 1.0) - mu * (mm_V0(x + 0.5 * h, 1.0) - mm_V0(x - 0.5 * h, 1.0));
        }
      }
    }
    B0[k] = b0;
    B1[k] = b1;
  }
  if (i < nx) {  // v face (i, j)
    const long long k = (long long)n * P + (long long)j * P + i;
    const double x = (i - iw + 0.5) * h, y = 1.0 + j * h;
    double b0 = 0.0, b1 = 0.0;
    if (!mms) {
    } else if (j == n) {
      b1 = mm_V0(x, 2.0);
    } else if (j == 0 && !on_gamma(c, i)) {
      b1 = mm_V0(x, 1.0);
    } else if (j == 0) {
      b0 = 0.5 * h2 * mm_V0(x, 1.0);
      b1 = 0.5 * h2 * mm_f1y(x, 1.0, mu);
      if (!on_gamma(c, i - 1)) b1 += 0.5 * h * c.w[i] * mm_V0(x - h, 1.0);
      if (!on_gamma(c, i + 1)) b1 += 0.5 * h * c.w[i + 1] * mm_V0(x + h, 1.0);
    } else {
      b0 = h2 * mm_V0(x, y);
      b1 = h2 * mm_f1y(x, y, mu);
      if (j == n - 1) b1 += 2.0 * mu * mm_V0(x, 2.0);
      if (j == 1 && !on_gamma(c, i)) b1 += 2.0 * mu * mm_V0(x, 1.0);
      if (i == 0) {
        if (lat) b1 += 2.0 * mu * mm_V0(xl, y);
        else b1 += 2.0 * mu * mm_V0(xl, y) - mu * (mm_U0(xl, y + 0.5 * h) - mm_U0(xl, y - 0.5 * h));
      }
      if (i == nx - 1) {
        if (lat) b1 += 2.0 * mu * mm_V0(xr, y);
        else b1 += 2.0 * mu * mm_V0(xr, y) + mu * (mm_U0(xr, y + 0.5 * h) - mm_U0(xr, y - 0.5 * h));
      }
    }
    B0[k] = b0;
    B1[k] = b1;
  }
  if (i < nx && j < n) {  // continuity
    const long long kc = (long long)j * P + i;
    const double y = 1.0 + (j + 0.5) * h, x = (i - iw + 0.5) * h;
    double s = 0.0;
    if (mms) {
      if (i == 0 && !lat) s += h * mm_U0(xl, y);
      if (i == nx - 1 && !lat) s -= h * mm_U0(xr, y);
      if (j == n - 1) s -= h * mm_V0(x, 2.0);
      if (j == 0 && !on_gamma(c, i)) s += h * mm_V0(x, 1.0);
    }
    B0[(long long)(2 * n + 1) * P + kc] = 0.0;
    B1[(long long)(2 * n + 1) * P + kc] = s;
  }
  if (i < n && j < n) {  // Darcy
    const long long kc = (long long)j * P + i;
    double sp = 0.0;
    if (j == 0 && mms) sp = 2.0 * K[i] / mu * mm_Ppm0((i + 0.5) * h, 0.0);
    B0[(long long)(3 * n + 1) * P + kc] = 0.0;
    B1[(long long)(3 * n + 1) * P + kc] = sp;
  }
}

void launch_mms_terms(const Coef<double>& c, int bc, const double* Kp, double* B0, double* B1, cudaStream_t s) {
  SD_COUNT(1);
  if (c.iw > 0)
    launch_k(k_mms_terms_ch, dim3(grid2(c.nx + 1, c.n + 1)), dim3(dim3(BX, BY)), 0, s, c, bc, Kp, B0, B1);
  else
    launch_k(k_mms_terms, dim3(grid2(c.n + 1, c.n + 1)), dim3(dim3(BX, BY)), 0, s, c, bc, Kp, B0, B1);
}

// the manufactured state; free-flow x of u face i is (i - iw) h
__global__ void k_mms_exact(int n, int nx, int iw, int P, double mu, double t, double* __restrict__ x) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > nx || j > n) return;
  const double h = 1.0 / n, s = 1.0 + t;
  if (j < n) x[(long long)j * P + i] = s * mm_U0((i - iw) * h, 1.0 + (j + 0.5) * h);
  if (i < nx) x[(long long)n * P + (long long)j * P + i] = s * mm_V0((i - iw + 0.5) * h, 1.0 + j * h);
  if (i < nx && j < n) x[(long long)(2 * n + 1) * P + (long long)j * P + i] = s * mm_Pff0((i - iw + 0.5) * h, mu);
  if (i < n && j < n) x[(long long)(3 * n + 1) * P + (long long)j * P + i] = s * mm_Ppm0((i + 0.5) * h, (j + 0.5) * h);
}

void launch_mms_exact(const Geom& g, double mu, double t, double* x, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_mms_exact, dim3(grid2(g.nx + 1, g.n + 1)), dim3(dim3(BX, BY)), 0, s, g.n, g.nx, g.iw, g.P, mu, t, x);
}

// b = mass * xprev + B0 + s1 * B1 (mass = h^2/dt on velocity rows, half on
// v_Gamma and on traction-side u faces, 0 elsewhere); Dirichlet rows of x
// take their new values.
__global__ void k_rhs(int n, int nx, int iw, int P, int lat, double cm, const double* __restrict__ B0,
                      const double* __restrict__ B1, double s1, const double* __restrict__ xprev,
                      double* __restrict__ b, double* __restrict__ x) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > nx || j > n) return;
  if (j < n) {
    const long long k = (long long)j * P + i;
    const bool side = (i == 0 || i == nx), dir = side && !lat;
    const double m = dir ? 0.0 : (side ? 0.5 * cm : cm);
    const double val = m * xprev[k] + B0[k] + s1 * B1[k];
    b[k] = val;
    if (dir) x[k] = val;
  }
  if (i < nx) {
    const long long k = (long long)n * P + (long long)j * P + i;
    // the lid and, in the channel, the floor beside the interface are Dirichlet
    const bool dir = (j == n) || (j == 0 && (i < iw || i >= iw + n));
    const double m = dir ? 0.0 : (j == 0 ? 0.5 * cm : cm);
    const double val = m * xprev[k] + B0[k] + s1 * B1[k];
    b[k] = val;
    if (dir) x[k] = val;
  }
  if (i < nx && j < n) {
    const long long kp = (long long)(2 * n + 1) * P + (long long)j * P + i;
    b[kp] = B0[kp] + s1 * B1[kp];
  }
  if (i < n && j < n) {
    const long long km = (long long)(3 * n + 1) * P + (long long)j * P + i;
    b[km] = B0[km] + s1 * B1[km];
  }
}

void launch_rhs(const Geom& g, int lat, double cm, const double* B0, const double* B1, double s1,
                const double* xprev, double* b, double* x, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_rhs, dim3(grid2(g.nx + 1, g.n + 1)), dim3(dim3(BX, BY)), 0, s, g.n, g.nx, g.iw, g.P, lat, cm, B0, B1,
           s1, xprev, b, x);
}

// ------------------------------------------------------------ pack/unpack
// canonical dense layout: u (nx+1) x n, v nx x (n+1), p_ff nx x n, p_pm n x n,
// x fastest (nx = n in the square geometry)
__global__ void k_pack2(int n, int nx, int P, const double* __restrict__ src, double* __restrict__ dst,
                        int to_padded) {
  griddep_wait();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > nx || j > n) return;
  const long long nu = (long long)n * (nx + 1), nv = (long long)nx * (n + 1), npf = (long long)nx * n;
  long long kd[4], kp[4];
  bool ok[4];
  ok[0] = j < n;           kd[0] = (long long)j * (nx + 1) + i;           kp[0] = (long long)j * P + i;
  ok[1] = i < nx;          kd[1] = nu + (long long)j * nx + i;            kp[1] = (long long)n * P + (long long)j * P + i;
  ok[2] = i < nx && j < n; kd[2] = nu + nv + (long long)j * nx + i;       kp[2] = (long long)(2 * n + 1) * P + (long long)j * P + i;
  ok[3] = i < n && j < n;  kd[3] = nu + nv + npf + (long long)j * n + i;  kp[3] = (long long)(3 * n + 1) * P + (long long)j * P + i;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (!ok[q]) continue;
    if (to_padded) dst[kp[q]] = src[kd[q]];
    else dst[kd[q]] = src[kp[q]];
  }
}

void launch_pack(const Geom& g, const double* dense, double* padded, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_pack2, dim3(grid2(g.nx + 1, g.n + 1)), dim3(dim3(BX, BY)), 0, s, g.n, g.nx, g.P, dense, padded, 1);
}
void launch_unpack(const Geom& g, const double* padded, double* dense, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_pack2, dim3(grid2(g.nx + 1, g.n + 1)), dim3(dim3(BX, BY)), 0, s, g.n, g.nx, g.P, padded, dense, 0);
}

// ------------------------------------------------------- instantiations
#define SD_INST(T)                                                                                               \
  template void launch_setup_coef<T>(const double*, int, int, int, double, double, int, int, int, int, int, int, \
                                     T*, T*, T*, T*, cudaStream_t);                                                \
  template void launch_convert<T>(const double*, T*, long long, cudaStream_t, const double*);                                   \
  template void launch_cheb_V<T>(const Coef<T>&, const T*, const T*, T*, T*, T, T, const T*, int, long long, cudaStream_t); \
  template void launch_cheb_D<T>(const Coef<T>&, const T*, const T*, T*, T*, T, T, const T*, int, long long, cudaStream_t); \
  template void launch_resid_V<T>(const Coef<T>&, const T*, const T*, T*, int, int, long long, cudaStream_t);    \
  template void launch_resid_D<T>(const Coef<T>&, const T*, const T*, T*, int, int, long long, cudaStream_t);    \
  template void launch_restrict_V<T>(int, int, const T*, int, int, int, int, T*, int, cudaStream_t);             \
  template void launch_restrict_D<T>(int, int, const T*, int, int, T*, cudaStream_t);            \
  template void launch_prolong_V<T>(int, int, T*, int, int, int, int, const T*, int, cudaStream_t);               \
  template void launch_prolong_D<T>(int, int, int, T*, int, int, const T*, cudaStream_t);                         \
  template void launch_resid_restrict_D<T>(const Coef<T>&, const T*, const T*, int, int, T*, cudaStream_t);                              \
  template void launch_precond_entry<T>(const Coef<double>&, const double*, double*, double, const T*, double, int, int, T*, cudaStream_t, const double*); \
  template void launch_precond_mid<T>(const Coef<double>&, const double*, double*, const T*, int, T*, cudaStream_t, const double*); \
  template void launch_precond_exit<T>(const Coef<double>&, double*, const T*, cudaStream_t);                     \
  template void launch_precond_bgs_pff<T>(const Coef<double>&, const double*, double*, const T*, cudaStream_t, const double*);
SD_INST(float)
SD_INST(double)
template int launch_coarse_cycle<float>(const CoarseCycle<float>&, cudaStream_t);
template int prepare_coarse_cycle<float>();
template int launch_smooth_tile_D<float>(const Coef<float>&, const float*, const float*, float*, const ChebSteps<float>&,
                                         const float*, const float*, int, int, cudaStream_t);
template int launch_smooth_tile_V<float>(const Coef<float>&, const float*, const float*, float*, const ChebSteps<float>&,
                                         const float*, const float*, int, int, cudaStream_t);
template int launch_smooth_tile_V_rr<float>(const Coef<float>&, const float*, float*, const ChebSteps<float>&,
                                             const float*, int, int, float*, cudaStream_t);
template int launch_smooth_tile_D_rr<float>(const Coef<float>&, const float*, float*, const ChebSteps<float>&,
                                             const float*, int, int, float*, cudaStream_t);
template int prepare_coarse_cycle<double>();
template int launch_coarse_cycle<double>(const CoarseCycle<double>&, cudaStream_t);
template size_t coarse_cycle_smem<float>(const CoarseCycle<float>&);
template size_t coarse_cycle_smem<double>(const CoarseCycle<double>&);

}  // namespace sdk
