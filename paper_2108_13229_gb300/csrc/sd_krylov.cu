// sd_krylov.cu -- FP64 kernels of the flexible GMRES(m) outer solve (the
// Krylov solver that replaces the paper's PD-GMRES, Sec. 5) and the dense
// coarsest-level solve of the multigrid V-cycles.
//
//  * multi-dot and fused update+dot kernels for classical Gram-Schmidt with
//    one re-orthogonalisation (CGS2): each block accumulates its slice of
//    all k dot products in registers, sums them over its threads in shared
//    memory and writes one partial per block; a one-block kernel per dot adds
//    the partials up in a fixed order, so every reduction is deterministic
//    (bitwise repeatable).  (Summing them in the block that finishes last
//    instead, one launch fewer, was measured slower: with programmatic
//    dependent launch the separate kernel's launch is hidden, while the
//    last-block count lengthens every block of the producer.)
//  * Givens rotations, residual estimate and back substitution on the
//    (m+1) x m Hessenberg matrix, kept on the device (one thread).
//  * dense coarse solve x = A_c^{-1} b with the inverse built at setup by a
//    Gauss-Jordan elimination with partial pivoting (one launch per column).
#include "sd_internal.cuh"

#include <math.h>

#include <algorithm>

namespace sdk {

std::atomic<long long> g_launch_count{0};
thread_local long long t_launch_count = 0;
thread_local int t_pdl = 0;
thread_local Bat t_bat = {nullptr, nullptr};
thread_local int t_bat_n = 1;
thread_local int t_bat_misuse = 0;

static const int RT = 256;       // threads per reduction / update block
static const int KT = 128;       // threads per Gram-Schmidt block
static const int KE = 16;        // vector elements owned by one Gram-Schmidt thread
static const int KMAX_REG = 32;  // max dot products per pass

// Blocks of the Gram-Schmidt kernels for a vector of length len: each block
// owns KT * KE consecutive elements (fixed for a given len, so every
// reduction sums its partials in the same order on every call).
int reduce_blocks(long long len) {
  long long nb = (len + (long long)KT * KE - 1) / ((long long)KT * KE);
  return (int)(nb < 1 ? 1 : nb);
}

// Per-thread dot of its KE elements: four interleaved partial sums.
__device__ __forceinline__ double own_dot(const double* __restrict__ v, const double* we, long long base,
                                          long long len) {
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll
  for (int t = 0; t < KE; t += 4) {
    const long long e = base + (long long)t * KT;
    if (e < len) s0 = fma(v[e], we[t], s0);
    if (e + KT < len) s1 = fma(v[e + KT], we[t + 1], s1);
    if (e + 2 * KT < len) s2 = fma(v[e + 2 * KT], we[t + 2], s2);
    if (e + 3 * KT < len) s3 = fma(v[e + 3 * KT], we[t + 3], s3);
  }
  return (s0 + s1) + (s2 + s3);
}

// red[q][tid] holds every thread's partial of dot q (q < kk); a fixed binary
// tree over tid (all q at once) leaves the block sum in red[q][0], written to
// partial[q * ps + block].
__device__ __forceinline__ void block_tree(double (*red)[KT], int kk, double* partial, int ps) {
  __syncthreads();
  for (int st = KT / 2; st > 0; st >>= 1) {
    for (int p = threadIdx.x; p < kk * st; p += KT) {
      const int q = p / st, t = p - q * st;
      red[q][t] += red[q][t + st];
    }
    __syncthreads();
  }
  if (threadIdx.x < kk) partial[(long long)threadIdx.x * ps + blockIdx.x] = red[threadIdx.x][0];
}

__device__ __forceinline__ void load_own(const double* __restrict__ w, double* we, long long base, long long len) {
#pragma unroll
  for (int t = 0; t < KE; ++t) {
    const long long e = base + (long long)t * KT;
    we[t] = e < len ? w[e] : 0.0;
  }
}

// partial[q * ps + blk] = the block's share of V_q . w, q < k (summed by
// k_reduce).  cond (may be null): skip when 0.
__global__ void __launch_bounds__(KT) k_mdot(const double* __restrict__ V, long long vs, int k,
                                             const double* __restrict__ w, long long len, double* __restrict__ partial,
                                             int ps, const double* __restrict__ cond, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    V = bsh(V, o);
    w = bsh(w, o);
    partial = bsh(partial, o);
    cond = bsh(cond, o);
  }
  if (cond && cond[0] == 0.0) return;
  __shared__ double red[KMAX_REG][KT];
  const long long base = (long long)blockIdx.x * KT * KE + threadIdx.x;
  double we[KE];
  load_own(w, we, base, len);
  int q = 0;
  for (; q + 1 < k; q += 2) {
    const double a0 = own_dot(V + (long long)q * vs, we, base, len);
    const double a1 = own_dot(V + (long long)(q + 1) * vs, we, base, len);
    red[q][threadIdx.x] = a0;
    red[q + 1][threadIdx.x] = a1;
  }
  if (q < k) red[q][threadIdx.x] = own_dot(V + (long long)q * vs, we, base, len);
  block_tree(red, k, partial, ps);
}

void launch_mdot(const double* V, long long vstride, int k, const double* w, long long len, double* partial, int ps,
                 int nblk, const double* cond, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_mdot, dim3(nblk), dim3(KT), 0, s, V, vstride, k, w, len, partial, ps, cond);
}

// w -= sum_q coef_q qs_q V_q (qs null: 1; the scales of basis vectors kept
// unnormalised), then partials (as k_mdot) of
//   mode 1: V_q . w, q < k (second Gram-Schmidt pass),
//   mode 2: w . w (norm of the new basis vector).
__global__ void __launch_bounds__(KT) k_mupdate(const double* __restrict__ V, long long vs, int k,
                                                const double* __restrict__ coef, double* __restrict__ w,
                                                long long len, double* __restrict__ partial, int ps, int mode,
                                                const double* __restrict__ cond, const double* __restrict__ qs,
                                                Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    V = bsh(V, o);
    coef = bsh(coef, o);
    w = bsh(w, o);
    partial = bsh(partial, o);
    cond = bsh(cond, o);
    qs = bsh(qs, o);
  }
  if (cond && cond[0] == 0.0) return;
  __shared__ double cf[KMAX_REG];
  __shared__ double red[KMAX_REG][KT];
  if (threadIdx.x < KMAX_REG)
    cf[threadIdx.x] = threadIdx.x < k ? (qs ? coef[threadIdx.x] * qs[threadIdx.x] : coef[threadIdx.x]) : 0.0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * KT * KE + threadIdx.x;
  double we[KE];
  load_own(w, we, base, len);
  int q = 0;
  for (; q + 1 < k; q += 2) {
    const double* v0 = V + (long long)q * vs;
    const double* v1 = V + (long long)(q + 1) * vs;
    const double c0 = cf[q], c1 = cf[q + 1];
#pragma unroll
    for (int t = 0; t < KE; ++t) {
      const long long e = base + (long long)t * KT;
      if (e < len) we[t] = fma(-c1, v1[e], fma(-c0, v0[e], we[t]));
    }
  }
  if (q < k) {
    const double* v0 = V + (long long)q * vs;
    const double c0 = cf[q];
#pragma unroll
    for (int t = 0; t < KE; ++t) {
      const long long e = base + (long long)t * KT;
      if (e < len) we[t] = fma(-c0, v0[e], we[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < KE; ++t) {
    const long long e = base + (long long)t * KT;
    if (e < len) w[e] = we[t];
  }
  if (mode == 1) {
    q = 0;
    for (; q + 1 < k; q += 2) {
      const double a0 = own_dot(V + (long long)q * vs, we, base, len);
      const double a1 = own_dot(V + (long long)(q + 1) * vs, we, base, len);
      red[q][threadIdx.x] = a0;
      red[q + 1][threadIdx.x] = a1;
    }
    if (q < k) red[q][threadIdx.x] = own_dot(V + (long long)q * vs, we, base, len);
    block_tree(red, k, partial, ps);
  } else {
    double s0 = 0.0, s1 = 0.0;
#pragma unroll
    for (int t = 0; t < KE; t += 2) {
      s0 = fma(we[t], we[t], s0);
      s1 = fma(we[t + 1], we[t + 1], s1);
    }
    red[0][threadIdx.x] = s0 + s1;
    block_tree(red, 1, partial, ps);
  }
}

void launch_mupdate(const double* V, long long vstride, int k, const double* coef, double* w, long long len,
                    double* partial, int ps, int nblk, int mode, const double* cond, cudaStream_t s,
                    const double* qs) {
  SD_COUNT(1);
  launch_k(k_mupdate, dim3(nblk), dim3(KT), 0, s, V, vstride, k, coef, w, len, partial, ps, mode, cond, qs);
}

// out[q] = sum_b partial[q * ps + b] (times qs[q] unless qs is null: the
// scale of basis vector q, kept unnormalised), q < k, one block per q in a
// fixed-order tree; cond (may be null): nothing when cond[0] == 0 (a skipped
// pass).
// With reo (k = 1, the norm w'.w' of the first pass's projected w): the
// re-orthogonalisation decision (Daniel-Gragg-Kaufman-Stewart), reo[0] = 1
// when w'.w' < eta2 ||w||^2, else 0, where ||w||^2 = sum_{i < k1} h1_i^2 +
// w'.w' (Pythagoras over the orthonormal basis: w = sum_i h1_i V_i + w'), so
// no separate norm of w before the projection is formed.
__global__ void k_reduce(const double* __restrict__ partial, int nblk, int k, int ps, double* __restrict__ out,
                         const double* __restrict__ cond, const double* __restrict__ qs, const double* __restrict__ h1,
                         int k1, double eta2, double* __restrict__ reo, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    partial = bsh(partial, o);
    out = bsh(out, o);
    cond = bsh(cond, o);
    qs = bsh(qs, o);
    h1 = bsh(h1, o);
    reo = bsh(reo, o);
  }
  __shared__ double sm[RT / 32];
  const int q = blockIdx.x;
  if (q >= k) return;
  if (cond && cond[0] == 0.0) return;
  const double* p = partial + (long long)q * ps;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += RT) s += p[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) t += sm[w];
    out[q] = qs ? t * qs[q] : t;
    if (reo) {
      double nw2 = 0.0;
      for (int i = 0; i < k1; ++i) nw2 = fma(h1[i], h1[i], nw2);
      nw2 += t;
      reo[0] = t < eta2 * nw2 ? 1.0 : 0.0;
    }
  }
}

void launch_reduce(const double* partial, int nblk, int k, int ps, double* out, const double* cond, cudaStream_t s,
                   const double* qs) {
  SD_COUNT(1);
  launch_k(k_reduce, dim3(k), dim3(RT), 0, s, partial, nblk, k, ps, out, cond, qs, (const double*)nullptr, 0, 0.0,
           (double*)nullptr);
}

void launch_reduce_decide(const double* partial, int nblk, double* out, const double* h1, int k1, double eta2,
                          double* reo, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_reduce, dim3(1), dim3(RT), 0, s, partial, nblk, 1, nblk, out, (const double*)nullptr,
           (const double*)nullptr, h1, k1, eta2, reo);
}

void launch_dot(const double* a, const double* b, long long len, double* partial, int nblk, double* out,
                cudaStream_t s) {
  launch_mdot(a, 0, 1, b, len, partial, nblk, nblk, nullptr, s);
  launch_reduce(partial, nblk, 1, nblk, out, nullptr, s);
}

// mode 0: y = sdev[0] * x ; mode 1: y = x / sqrt(sdev[0])
__global__ void k_scale_by(const double* __restrict__ x, double* __restrict__ y, long long len,
                           const double* __restrict__ sdev, int mode, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    x = bsh(x, o);
    y = bsh(y, o);
    sdev = bsh(sdev, o);
  }
  const double f = mode == 0 ? sdev[0] : 1.0 / sqrt(sdev[0]);
  // 32-bit indices (a vector has fewer than 2^31 entries)
  const int n = (int)len;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) y[e] = f * x[e];
}

void launch_scale_by(const double* x, double* y, long long len, const double* sdev, int mode, cudaStream_t s) {
  SD_COUNT(1);
  const long long nb = (len + RT - 1) / RT;
  launch_k(k_scale_by, dim3((int)(nb < 152 * 16 ? nb : 152 * 16)), dim3(RT), 0, s, x, y, len, sdev, mode);
}

// x += sum_q y_q Z_q
__global__ void __launch_bounds__(KT) k_axpy_multi(double* __restrict__ x, const double* __restrict__ Z, long long zs,
                                                   const double* __restrict__ y, int k, long long len,
                                                   const double* __restrict__ kdev, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    x = bsh(x, o);
    Z = bsh(Z, o);
    y = bsh(y, o);
  }
  if (kdev) k = (int)bsh(kdev, o)[0];
  __shared__ double cf[KMAX_REG];
  if (threadIdx.x < KMAX_REG) cf[threadIdx.x] = threadIdx.x < k ? y[threadIdx.x] : 0.0;
  __syncthreads();
  const long long base = (long long)blockIdx.x * KT * KE + threadIdx.x;
  double xe[KE];
  load_own(x, xe, base, len);
  int q = 0;
  for (; q + 1 < k; q += 2) {
    const double* z0 = Z + (long long)q * zs;
    const double* z1 = Z + (long long)(q + 1) * zs;
    const double c0 = cf[q], c1 = cf[q + 1];
#pragma unroll
    for (int t = 0; t < KE; ++t) {
      const long long e = base + (long long)t * KT;
      if (e < len) xe[t] = fma(c1, z1[e], fma(c0, z0[e], xe[t]));
    }
  }
  if (q < k) {
    const double* z0 = Z + (long long)q * zs;
    const double c0 = cf[q];
#pragma unroll
    for (int t = 0; t < KE; ++t) {
      const long long e = base + (long long)t * KT;
      if (e < len) xe[t] = fma(c0, z0[e], xe[t]);
    }
  }
#pragma unroll
  for (int t = 0; t < KE; ++t) {
    const long long e = base + (long long)t * KT;
    if (e < len) x[e] = xe[t];
  }
}

void launch_axpy_multi(double* x, const double* Z, long long zstride, const double* ycoef, int k, long long len,
                       const double* kdev, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_axpy_multi, dim3(reduce_blocks(len)), dim3(KT), 0, s, x, Z, zstride, ycoef, k, len, kdev);
}

// ----------------------------------------------------- Hessenberg / Givens
// State layout (doubles): R[(m+1)*m] column-major (column j at j*(m+1)),
// cs[m], sn[m], g[m+1].  flag[0] = |g_{j+1}| (residual estimate),
// flag[1] = 1 / h_{j+1,j} (scale of the next basis vector), flag[2] = 1 on
// NaN/Inf, flag[3] = 1 on breakdown (h_{j+1,j} == 0).
__global__ void k_init_cycle(double* st, int m, const double* beta2, double* flag, double* vsc, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  st = bsh(st, o);
  beta2 = bsh(beta2, o);
  flag = bsh(flag, o);
  vsc = bsh(vsc, o);
  if (threadIdx.x != 0) return;
  double* g = st + (m + 1) * m + 2 * m;
  const double beta = sqrt(beta2[0]);
  g[0] = beta;
  for (int i = 1; i <= m; ++i) g[i] = 0.0;
  flag[0] = beta;
  flag[1] = beta > 0.0 ? 1.0 / beta : 0.0;
  flag[2] = isfinite(beta) ? 0.0 : 1.0;
  flag[3] = 0.0;
  flag[5] = 0.0;
  if (vsc) vsc[0] = flag[1];
}

void launch_init_cycle(double* st, int m, const double* beta2, double* flag, cudaStream_t s, double* vsc) {
  SD_COUNT(1);
  launch_k(k_init_cycle, dim3(1), dim3(32), 0, s, st, m, beta2, flag, vsc);
}

__global__ void k_givens(double* st, int j, int m, const double* h1, const double* h2, const double* nrm2a,
                         const double* nrm2b, const double* reo, double* flag, double* vsc, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (threadIdx.x != 0) return;
  if (bt.off) {
    st = bsh(st, o);
    h1 = bsh(h1, o);
    h2 = bsh(h2, o);
    nrm2a = bsh(nrm2a, o);
    nrm2b = bsh(nrm2b, o);
    reo = bsh(reo, o);
    flag = bsh(flag, o);
    vsc = bsh(vsc, o);
  }
  const bool second = reo == nullptr || reo[0] != 0.0;
  const double* nrm2 = second ? nrm2b : nrm2a;
  double* R = st;
  double* cs = st + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  double* col = R + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = second ? h1[i] + h2[i] : h1[i];
  const double hn = sqrt(nrm2[0]);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double a = col[i], b = col[i + 1];
    col[i] = cs[i] * a + sn[i] * b;
    col[i + 1] = -sn[i] * a + cs[i] * b;
  }
  const double a = col[j], b = col[j + 1];
  const double r = hypot(a, b);
  double c = 1.0, s = 0.0;
  if (r > 0.0) { c = a / r; s = b / r; }
  cs[j] = c;
  sn[j] = s;
  col[j] = r;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  flag[0] = fabs(g[j + 1]);
  flag[1] = hn > 0.0 ? 1.0 / hn : 0.0;
  flag[2] = (isfinite(r) && isfinite(g[j + 1])) ? 0.0 : 1.0;
  flag[3] = hn > 0.0 ? 0.0 : 1.0;
  flag[4] = second ? 1.0 : 0.0;
  flag[5] = (double)(j + 1);
  if (vsc) vsc[j + 1] = flag[1];
}

void launch_givens(double* st, int j, int m, const double* hcol1, const double* hcol2, const double* nrm2a,
                   const double* nrm2b, const double* reo, double* flag, cudaStream_t s, double* vsc) {
  SD_COUNT(1);
  launch_k(k_givens, dim3(1), dim3(32), 0, s, st, j, m, hcol1, hcol2, nrm2a, nrm2b, reo, flag, vsc);
}

// Polynomial extrapolation in time over the known levels: the history shifts
// (x3 <- x_mm, x_mm <- x_m, x_m <- x; x_mm and x3 may be null) and x becomes
// the extrapolation of the given order: 0: x (no extrapolation); 1: 2 x - x_m;
// 2: 3 x - 3 x_m + x_mm; 3: 4 x - 6 x_m + 4 x_mm - x3.  The order never
// exceeds the history the caller holds (x_mm for 2, x3 for 3).
__global__ void k_extrapolate(double* __restrict__ x, double* __restrict__ xm, double* __restrict__ xmm,
                               double* __restrict__ x3, long long len, int order) {
  griddep_wait();
  const int n = (int)len;  // 32-bit indices: fewer than 2^31 entries
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const double t = x[e], m = xm[e], mm = xmm ? xmm[e] : 0.0;
    x[e] = order >= 3 ? 4.0 * (t + mm) - 6.0 * m - x3[e] : order == 2 ? 3.0 * (t - m) + mm
                                                         : order == 1 ? 2.0 * t - m : t;
    if (x3) x3[e] = mm;
    if (xmm) xmm[e] = m;
    xm[e] = t;
  }
}

void launch_extrapolate(double* x, double* xm, double* xmm, double* x3, long long len, int order, cudaStream_t s) {
  SD_COUNT(1);
  const long long nb = (len + RT - 1) / RT;
  launch_k(k_extrapolate, dim3((int)(nb < 152 * 16 ? nb : 152 * 16)), dim3(RT), 0, s, x, xm, xmm, x3, len, order);
}

// The operator applied to the extrapolated initial guess, from the history of
// the operator applied to the solved states (the extrapolation is a linear
// combination, so A x^0 is the same combination of the A x^{n-i}): Y0 =
// A x^n (stored by the last solve's residual), Y1 = A x^{n-1}, ... (Y1..Y3
// may be null, the depth the handle keeps).  With use != 0, r = A x^0 by the
// extrapolation of the given order, the same arithmetic as k_extrapolate's
// on the states; then the history shifts (Y1 <- Y0, ...; Y0 receives the
// step's own A x).  rh[0] = use: the step's first residual is b - r
// (k_resid_hist) instead of an operator application.
__global__ void k_yhist(double* __restrict__ Y0, double* __restrict__ Y1, double* __restrict__ Y2,
                        double* __restrict__ Y3, double* __restrict__ r, long long len, int order, int use,
                        double* __restrict__ rh) {
  griddep_wait();
  if (blockIdx.x == 0 && threadIdx.x == 0) rh[0] = use ? 1.0 : 0.0;
  const int n = (int)len;  // 32-bit indices: fewer than 2^31 entries
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const double t = Y0[e], m = Y1 ? Y1[e] : 0.0, mm = Y2 ? Y2[e] : 0.0, m3 = Y3 ? Y3[e] : 0.0;
    if (use)
      r[e] = order >= 3 ? 4.0 * (t + mm) - 6.0 * m - m3 : order == 2 ? 3.0 * (t - m) + mm
                                                      : order == 1 ? 2.0 * t - m : t;
    if (Y3) Y3[e] = mm;
    if (Y2) Y2[e] = m;
    if (Y1) Y1[e] = t;
  }
}

void launch_yhist(double* const* Y, int depth, double* r, long long len, int order, int use, double* rh,
                  cudaStream_t s) {
  SD_COUNT(1);
  const long long nb = (len + RT - 1) / RT;
  launch_k(k_yhist, dim3((int)(nb < 152 * 16 ? nb : 152 * 16)), dim3(RT), 0, s, Y[0], depth > 1 ? Y[1] : nullptr,
           depth > 2 ? Y[2] : nullptr, depth > 3 ? Y[3] : nullptr, r, len, order, use, rh);
}

__global__ void k_backsolve(const double* st, int k, int m, double* y, const double* kdev, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (threadIdx.x != 0) return;
  if (bt.off) {
    st = bsh(st, o);
    y = bsh(y, o);
  }
  if (kdev) k = (int)bsh(kdev, o)[0];
  const double* R = st;
  const double* g = st + (m + 1) * m + 2 * m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= R[(long long)l * (m + 1) + i] * y[l];
    y[i] = s / R[(long long)i * (m + 1) + i];
  }
}

void launch_backsolve(double* st, int k, int m, double* y, const double* kdev, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_backsolve, dim3(1), dim3(32), 0, s, st, k, m, y, kdev);
}

// ------------------------------------------------ device-side loop control
// With graph option 2 a whole FGMRES solve is one CUDA graph: the restart
// loop is a WHILE node and the m Arnoldi steps of a cycle a chain of IF
// nodes.  These one-thread kernels take the decisions that the host takes
// between graph replays otherwise, on the same FP64 values and in the same
// order, so both paths run the same iterations (layout of ctl in
// sd_internal.cuh).  Every control kernel also adds the number of kernels
// of the graph segment it closes to ctl[C_KERN].

// ||b|| and the tolerances; counters cleared (accept <= 0: no acceptance of
// a stagnating solve)
__global__ void k_solve_begin(const double* bn2, double rtol, double accept, double* ctl) {
  griddep_wait();
  if (threadIdx.x != 0) return;
  const double bnorm = sqrt(bn2[0]);
  const double bs = bnorm > 0 ? bnorm : 1.0;
  ctl[C_TOL] = rtol * bs;
  ctl[C_ACC] = accept > 0 ? accept * bs : -1.0;
  ctl[C_BN] = bnorm;
  ctl[C_ITER] = ctl[C_REST] = ctl[C_REO] = ctl[C_STAT] = ctl[C_KERN] = 0.0;
  ctl[C_REL] = ctl[C_PREV] = 0.0;
}

// after a true residual: stop (converged, NaN/Inf, budget spent, a NaN
// inside the last cycle, or a cycle that did not halve the residual when
// stagnation is accepted) or start another cycle
__global__ void k_restart_ctrl(const double* beta2, double* ctl, int max_iters, double kern,
                               cudaGraphConditionalHandle loop) {
  griddep_wait();
  if (threadIdx.x != 0) return;
  const double beta = sqrt(beta2[0]);
  const double bn = ctl[C_BN];
  const double prev = ctl[C_PREV];
  ctl[C_PREV] = beta;
  ctl[C_REL] = bn > 0 ? beta / bn : beta;
  ctl[C_KERN] += kern;
  bool go = false;
  if (ctl[C_STAT] != 0.0) {
  } else if (!isfinite(beta)) {
    ctl[C_STAT] = C_STAT_NUMERIC;
  } else if (beta <= ctl[C_TOL]) {
  } else if (ctl[C_ACC] >= 0.0 && ctl[C_REST] > 0.0 && beta > 0.5 * prev) {
    if (beta > ctl[C_ACC]) ctl[C_STAT] = C_STAT_NOCONV;
  } else if (ctl[C_ITER] >= (double)max_iters) {
    ctl[C_STAT] = C_STAT_NOCONV;
  } else {
    go = true;
    ctl[C_REST] += 1.0;
  }
  cudaGraphSetConditional(loop, go ? 1u : 0u);
}

// start of a cycle: no Arnoldi step after the first runs unless the step
// before it says so (the IF handles keep their value across WHILE iterations)
__global__ void k_cycle_head(CondSet cs) {
  griddep_wait();
  if (threadIdx.x != 0) return;
  for (int i = 2; i < cs.n; ++i) cudaGraphSetConditional(cs.c[i], 0u);
}

// after Arnoldi step j: count it, and run step j + 1 unless the residual
// estimate is below the tolerance, the step broke down or hit NaN/Inf, or the
// iteration budget is spent; a NaN/Inf drops the cycle's update of x
// (k = flag[5] = 0)
__global__ void k_step_ctrl(double* flag, double* ctl, int max_iters, double kern, int has_next,
                            cudaGraphConditionalHandle next) {
  griddep_wait();
  if (threadIdx.x != 0) return;
  const double it = ctl[C_ITER] + 1.0;
  ctl[C_ITER] = it;
  ctl[C_REO] += flag[4] != 0.0 ? 1.0 : 0.0;
  ctl[C_KERN] += kern;
  const bool numeric = flag[2] != 0.0;
  if (numeric) {
    flag[5] = 0.0;
    ctl[C_STAT] = C_STAT_NUMERIC;
  }
  const bool stop = numeric || flag[0] <= ctl[C_TOL] || flag[3] != 0.0 || it >= (double)max_iters;
  if (has_next) cudaGraphSetConditional(next, stop ? 0u : 1u);
}

void launch_solve_begin(const double* bn2, double rtol, double accept, double* ctl, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_solve_begin, dim3(1), dim3(32), 0, s, bn2, rtol, accept, ctl);
}
void launch_restart_ctrl(const double* beta2, double* ctl, int max_iters, double kern,
                         cudaGraphConditionalHandle loop, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_restart_ctrl, dim3(1), dim3(32), 0, s, beta2, ctl, max_iters, kern, loop);
}
void launch_cycle_head(const CondSet& cs, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_cycle_head, dim3(1), dim3(32), 0, s, cs);
}
void launch_step_ctrl(double* flag, double* ctl, int max_iters, double kern, int has_next,
                      cudaGraphConditionalHandle next, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_step_ctrl, dim3(1), dim3(32), 0, s, flag, ctl, max_iters, kern, has_next, next);
}

// ------------------------------------------- lockstep groups in one graph
// The host-driven lockstep (fgmres_lockstep) decides, after each true
// residual and each Arnoldi step, which instances of the group go on.  These
// kernels take the same decisions on the same FP64 values, per instance, on
// the device, so a group's whole solve runs inside a CUDA graph (WHILE / IF
// nodes) with every instance doing the arithmetic of its solo run.
__global__ void k_grp_act_all(int* act, int B) {
  griddep_wait();
  for (int z = threadIdx.x; z < B; z += blockDim.x) act[z] = 1;
}

__global__ void k_grp_begin(const long long* __restrict__ off, int B, const double* bn2, double* ctl0, double rtol) {
  griddep_wait();
  for (int z = threadIdx.x; z < B; z += blockDim.x) {
    double* ctl = bsh(ctl0, off[z]);
    const double bn = sqrt(bsh(bn2, off[z])[0]);
    ctl[C_TOL] = rtol * (bn > 0 ? bn : 1.0);
    ctl[C_BN] = bn;
    ctl[C_ITER] = ctl[C_REST] = ctl[C_REO] = ctl[C_STAT] = ctl[C_REL] = ctl[C_PREV] = 0.0;
    ctl[C_ACC] = -1.0;
    ctl[C_LIVE] = 1.0;
    ctl[C_CYC] = ctl[C_NUMR] = 0.0;
  }
  if (threadIdx.x == 0) ctl0[C_KERN] = ctl0[C_GCYC] = 0.0;  // instance 0's slots sit at offset 0
}

__global__ void k_grp_restart(const long long* __restrict__ off, int* act, int B, const double* b2, double* ctl0,
                              int max_iters, int max_cycles, double kern, cudaGraphConditionalHandle loop) {
  griddep_wait();
  // a bound on the device loop: every cycle adds at least one iteration to
  // each instance that takes part, so max_iters cycles are never exceeded
  const bool capped = ctl0[C_GCYC] >= (double)max_cycles;
  int any = 0;
  for (int z = threadIdx.x; z < B; z += blockDim.x) {
    double* ctl = bsh(ctl0, off[z]);
    int cyc = 0;
    if (ctl[C_LIVE] != 0.0) {
      const double beta = sqrt(bsh(b2, off[z])[0]);
      const double bn = ctl[C_BN];
      ctl[C_REL] = bn > 0 ? beta / bn : beta;
      if (!isfinite(beta)) {
        ctl[C_STAT] = C_STAT_NUMERIC;
        ctl[C_LIVE] = 0.0;
      } else if (beta <= ctl[C_TOL]) {
        ctl[C_LIVE] = 0.0;
      } else if (ctl[C_ITER] >= (double)max_iters || capped) {
        ctl[C_STAT] = C_STAT_NOCONV;
        ctl[C_LIVE] = 0.0;
      } else {
        cyc = 1;
        ctl[C_REST] += 1.0;
      }
    }
    ctl[C_CYC] = cyc;
    act[z] = cyc;
    any |= cyc;
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    ctl0[C_KERN] += kern;
    if (any) ctl0[C_GCYC] += 1.0;
    cudaGraphSetConditional(loop, any ? 1u : 0u);
  }
}

__global__ void k_grp_step(const long long* __restrict__ off, int* act, int B, const double* flag0, double* ctl0,
                           int max_iters, double kern, int has_next, cudaGraphConditionalHandle next) {
  griddep_wait();
  int running = 0;
  for (int z = threadIdx.x; z < B; z += blockDim.x) {
    if (!act[z]) continue;
    double* ctl = bsh(ctl0, off[z]);
    const double* f = bsh(flag0, off[z]);
    ctl[C_ITER] += 1.0;
    ctl[C_REO] += f[4] != 0.0 ? 1.0 : 0.0;
    if (f[2] != 0.0) {
      ctl[C_NUMR] = 1.0;
      act[z] = 0;
    } else if (f[0] <= ctl[C_TOL] || f[3] != 0.0 || ctl[C_ITER] >= (double)max_iters) {
      act[z] = 0;
    } else {
      running = 1;
    }
  }
  running = __syncthreads_or(running);
  if (threadIdx.x == 0) {
    ctl0[C_KERN] += kern;
    if (has_next) cudaGraphSetConditional(next, running ? 1u : 0u);
  }
}

__global__ void k_grp_cycle_end(const long long* __restrict__ off, int* act, int B, double* ctl0, double kern) {
  griddep_wait();
  for (int z = threadIdx.x; z < B; z += blockDim.x) {
    double* ctl = bsh(ctl0, off[z]);
    if (ctl[C_NUMR] != 0.0) {
      ctl[C_STAT] = C_STAT_NUMERIC;
      ctl[C_LIVE] = 0.0;
      ctl[C_CYC] = 0.0;
    }
    act[z] = ctl[C_CYC] != 0.0 ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) ctl0[C_KERN] += kern;
}

__global__ void k_grp_live(const long long* __restrict__ off, int* act, int B, const double* ctl0) {
  griddep_wait();
  for (int z = threadIdx.x; z < B; z += blockDim.x) act[z] = bsh(ctl0, off[z])[C_LIVE] != 0.0 ? 1 : 0;
}

void launch_grp_act_all(int* act, int B, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_act_all, dim3(1), dim3(256), 0, s, act, B);
}
void launch_grp_begin(const long long* off, int B, const double* bn2, double* ctl0, double rtol, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_begin, dim3(1), dim3(256), 0, s, off, B, bn2, ctl0, rtol);
}
void launch_grp_restart(const long long* off, int* act, int B, const double* b2, double* ctl0, int max_iters,
                        int max_cycles, double kern, cudaGraphConditionalHandle loop, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_restart, dim3(1), dim3(256), 0, s, off, act, B, b2, ctl0, max_iters, max_cycles, kern, loop);
}
void launch_grp_step(const long long* off, int* act, int B, const double* flag0, double* ctl0, int max_iters,
                     double kern, int has_next, cudaGraphConditionalHandle next, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_step, dim3(1), dim3(256), 0, s, off, act, B, flag0, ctl0, max_iters, kern, has_next, next);
}
void launch_grp_cycle_end(const long long* off, int* act, int B, double* ctl0, double kern, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_cycle_end, dim3(1), dim3(256), 0, s, off, act, B, ctl0, kern);
}
void launch_grp_live(const long long* off, int* act, int B, const double* ctl0, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_grp_live, dim3(1), dim3(256), 0, s, off, act, B, ctl0);
}

// out[z * count + t] = src_z[t] for every instance z of a lockstep batch
// (src moved to instance z; out is not), idle instances included
__global__ void k_gather_inst(const double* __restrict__ src, int count, double* __restrict__ out, Bat bt) {
  griddep_wait();
  const long long o = bt.off ? bt.off[blockIdx.z] : 0;
  const double* p = bsh(src, o);
  for (int t = threadIdx.x; t < count; t += blockDim.x) out[(long long)blockIdx.z * count + t] = p[t];
}

void launch_gather_inst(const double* src, int count, double* out, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_gather_inst, dim3(1), dim3(32), 0, s, src, count, out);
}

// ------------------------------------------------- IQN-ILS (partitioned, Sec. 3)
// One CTA updates the interface velocity of the partitioned coupling: the
// interface vectors have n entries (one per interface face), far too few to
// fill the GPU, and every step depends on the one before.  Sums use a fixed
// reduction order (warp shuffles, then the warps in order).

// sum over the block of one value per thread; red holds 33 doubles
__device__ double cta_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    red[32] = t;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

__device__ double cta_dot(const double* a, const double* b, int n, double* red) {
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[i], b[i], s);
  return cta_sum(s, red);
}

// Orthogonalise difference column c of st.Vc (copied to Q column q) against
// Q columns 0..q-1 (two Gram-Schmidt passes, projections added into R column
// q); keeps it as Q column q when it is not numerically dependent.  Returns
// the new column count.
__device__ int iqn_append(const IqnState& st, int c, int q, double* red) {
  const int n = st.n;
  double* Vq = st.Vc + (long long)q * st.ld;
  double* Wq = st.Wc + (long long)q * st.ld;
  double* qq = st.Q + (long long)q * st.ld;
  if (c != q) {
    const double* Vs = st.Vc + (long long)c * st.ld;
    const double* Ws = st.Wc + (long long)c * st.ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      Vq[i] = Vs[i];
      Wq[i] = Ws[i];
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) qq[i] = Vq[i];
  double* Rc = st.R + (long long)q * st.qmax;
  for (int l = threadIdx.x; l <= q; l += blockDim.x) Rc[l] = 0.0;
  __syncthreads();
  const double n0 = sqrt(cta_dot(qq, qq, n, red));
  for (int pass = 0; pass < 2; ++pass)
    for (int l = 0; l < q; ++l) {
      const double* ql = st.Q + (long long)l * st.ld;
      const double cl = cta_dot(ql, qq, n, red);
      for (int i = threadIdx.x; i < n; i += blockDim.x) qq[i] -= cl * ql[i];
      if (threadIdx.x == 0) Rc[l] += cl;
      __syncthreads();
    }
  const double nr = sqrt(cta_dot(qq, qq, n, red));
  if (!(nr > 1e-13 * n0)) return q;  // dependent on the kept columns (or zero): dropped
  const double inv = 1.0 / nr;
  for (int i = threadIdx.x; i < n; i += blockDim.x) qq[i] *= inv;
  if (threadIdx.x == 0) Rc[q] = nr;
  __syncthreads();
  return q + 1;
}

__global__ void __launch_bounds__(1024) k_iqn(IqnState st, const double* __restrict__ vt, const double* __restrict__ p) {
  griddep_wait();
  __shared__ double red[33];
  __shared__ double alpha[32];
  const int n = st.n;
  const int k = (int)st.scal[0];
  int q = (int)st.scal[1];
  double* v = st.v;
  // stopping test of Sec. 3: changes of the exchanged pressure and velocity
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double dp = p[i] - st.p_prev[i], dv = vt[i] - v[i];
    a0 = fma(dp, dp, a0);
    a1 = fma(p[i], p[i], a1);
    a2 = fma(dv, dv, a2);
    a3 = fma(vt[i], vt[i], a3);
  }
  const double s0 = cta_sum(a0, red), s1 = cta_sum(a1, red), s2 = cta_sum(a2, red), s3 = cta_sum(a3, red);
  if (threadIdx.x == 0) {
    st.scal[2] = k == 0 ? -1.0 : s0;  // no previous pressure yet
    st.scal[3] = s1;
    st.scal[4] = s2;
    st.scal[5] = s3;
  }
  if (k == 0) {  // relaxed first step
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const double r = vt[i] - v[i];
      st.r_prev[i] = r;
      st.vt_prev[i] = vt[i];
      st.p_prev[i] = p[i];
      v[i] = fma(st.omega0, r, v[i]);
    }
  } else {
    if (q == st.qmax) {  // drop the oldest difference and rebuild the factorisation
      int kept = 0;
      for (int c = 1; c < q; ++c) kept = iqn_append(st, c, kept, red);
      q = kept;
    }
    // new differences dr = r_k - r_{k-1}, dv~ = v~_k - v~_{k-1} as column q
    double* Vq = st.Vc + (long long)q * st.ld;
    double* Wq = st.Wc + (long long)q * st.ld;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      Vq[i] = (vt[i] - v[i]) - st.r_prev[i];
      Wq[i] = vt[i] - st.vt_prev[i];
    }
    __syncthreads();
    q = iqn_append(st, q, q, red);
    // alpha = argmin ||V alpha + r_k||: R alpha = -Q^T r_k
    for (int l = 0; l < q; ++l) {
      const double* ql = st.Q + (long long)l * st.ld;
      double s = 0.0;
      for (int i = threadIdx.x; i < n; i += blockDim.x) s = fma(ql[i], vt[i] - v[i], s);
      s = cta_sum(s, red);
      if (threadIdx.x == 0) alpha[l] = -s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int i = q - 1; i >= 0; --i) {
        double s = alpha[i];
        for (int l = i + 1; l < q; ++l) s -= st.R[(long long)l * st.qmax + i] * alpha[l];
        alpha[i] = s / st.R[(long long)i * st.qmax + i];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double vn = vt[i];
      for (int l = 0; l < q; ++l) vn = fma(alpha[l], st.Wc[(long long)l * st.ld + i], vn);
      st.r_prev[i] = vt[i] - v[i];
      st.vt_prev[i] = vt[i];
      st.p_prev[i] = p[i];
      v[i] = vn;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    st.scal[0] = (double)(k + 1);
    st.scal[1] = (double)q;
  }
}

void launch_iqn(const IqnState& st, const double* vt, const double* p, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_iqn, dim3(1), dim3(1024), 0, s, st, vt, p);
}

// ------------------------------------------------------ dense coarse solve
// x[idx[r]] = T(sum_l Ainv[r][l] b[idx[l]]): one warp per row r, its lanes
// striding over l, a fixed shuffle tree; the rows spread over as many CTAs
// as there are rows / 8 (each CTA stages b in shared memory), so a 544-row
// coarsest solve is not serialised on one SM's FP64 pipe.  Every row sums
// in the same order as in the single-CTA form of the fused coarse cycle.
template <typename T>
__global__ void k_dense_solve(const double* __restrict__ Ainv, const int* __restrict__ idx, int m,
                              const T* __restrict__ b, T* __restrict__ x, Bat bt) {
  griddep_wait();
  long long o;
  if (!bat_enter(bt, o)) return;
  if (bt.off) {
    Ainv = bsh(Ainv, o);
    idx = bsh(idx, o);
    b = bsh(b, o);
    x = bsh(x, o);
  }
  extern __shared__ double bs[];
  for (int l = threadIdx.x; l < m; l += blockDim.x) bs[l] = (double)b[idx[l]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = blockIdx.x * nw + warp; r < m; r += gridDim.x * nw) {
    const double* row = Ainv + (long long)r * m;
    double s = 0.0;
    for (int l = lane; l < m; l += 32) s = fma(row[l], bs[l], s);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[idx[r]] = (T)s;
  }
}

template <typename T>
void launch_dense_solve(const double* Ainv, const int* idx, int m, const T* b, T* x, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_dense_solve<T>, dim3((m + 7) / 8), dim3(256), sizeof(double) * m, s, Ainv, idx, m, b, x);
}

// Gauss-Jordan with partial pivoting on [A | I]; the inverse ends in W.
// Column c: the pivot step picks the pivot row (the largest |A[r][c]|,
// r >= c, the lowest r on ties), swaps it into row c, scales row c and
// records the elimination factors fc[r] = A[r][c] (0 for r = c); the
// elimination (all SMs) subtracts fc[r] times row c from every other row.
// The pivot step of column c + 1 is done by the last block of column c's
// elimination to finish (a completion counter, no waiting), so a column takes
// one launch.  A zero pivot sets *status = c + 1 and the remaining launches do
// nothing.  (One CTA for the whole elimination serialised 2m^3 FP64
// operations on one SM: 0.15 s for the 544-row coarsest velocity block.)
__global__ void k_gj_init(double* W, int m, int* status, int* counter) {
  griddep_wait();
  const long long mm = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mm; e += (long long)gridDim.x * blockDim.x)
    W[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *status = 0;
    *counter = 0;
  }
}

// the pivot step of column c by the calling block (any multiple of 32 threads
// up to 1024).  Its reads of A and W bypass L1 (ld.global.cg): called at the
// end of an elimination, it reads rows that other blocks have just written.
__device__ void gj_pivot_step(double* A, double* W, int m, int c, double* fc, int* status) {
  __shared__ double sbest[32];
  __shared__ int srow[32];
  __shared__ int piv;
  __shared__ double pval;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  // strided scan in increasing r keeps the first maximum, as does the tree
  double best = -1.0;
  int br = m;
  for (int r = c + tid; r < m; r += nt) {
    const double a = fabs(__ldcg(&A[(long long)r * m + c]));
    if (a > best) { best = a; br = r; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ob = __shfl_down_sync(0xffffffffu, best, o);
    const int orr = __shfl_down_sync(0xffffffffu, br, o);
    if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
  }
  if (lane == 0) { sbest[warp] = best; srow[warp] = br; }
  __syncthreads();
  if (tid == 0) {
    double b = sbest[0];
    int r = srow[0];
    for (int w = 1; w < (nt + 31) / 32; ++w)
      if (sbest[w] > b || (sbest[w] == b && srow[w] < r)) { b = sbest[w]; r = srow[w]; }
    piv = r;
    pval = b;
    if (!(b > 0.0)) *status = c + 1;
  }
  __syncthreads();
  if (!(pval > 0.0)) return;
  const int p = piv;
  if (p != c)
    for (int q = tid; q < m; q += nt) {
      const double ac = __ldcg(&A[(long long)c * m + q]), ap = __ldcg(&A[(long long)p * m + q]);
      A[(long long)c * m + q] = ap;
      A[(long long)p * m + q] = ac;
      const double wc = __ldcg(&W[(long long)c * m + q]), wp = __ldcg(&W[(long long)p * m + q]);
      W[(long long)c * m + q] = wp;
      W[(long long)p * m + q] = wc;
    }
  __syncthreads();
  const double inv = 1.0 / __ldcg(&A[(long long)c * m + c]);
  __syncthreads();
  for (int q = tid; q < m; q += nt) {
    A[(long long)c * m + q] = __ldcg(&A[(long long)c * m + q]) * inv;
    W[(long long)c * m + q] = __ldcg(&W[(long long)c * m + q]) * inv;
  }
  __syncthreads();
  for (int r = tid; r < m; r += nt) fc[r] = (r == c) ? 0.0 : __ldcg(&A[(long long)r * m + c]);
}

__global__ void __launch_bounds__(1024) k_gj_pivot(double* A, double* W, int m, int c, double* fc, int* status) {
  griddep_wait();
  if (*status != 0) return;
  gj_pivot_step(A, W, m, c, fc, status);
}

__global__ void __launch_bounds__(256) k_gj_eliminate(double* A, double* W, int m, int c, double* fc, int* status,
                                                      int* counter) {
  griddep_wait();
  if (*status != 0) return;  // uniform: no block goes on, none counts
  const long long mm = (long long)m * m;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < mm; e += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(e / m), q = (int)(e % m);
    const double f = fc[r];
    if (f != 0.0) {
      A[e] -= f * A[(long long)c * m + q];
      W[e] -= f * W[(long long)c * m + q];
    }
  }
  // the last block to finish takes the pivot step of the next column
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const int done = atomicAdd(counter, 1);
    last = done == (int)gridDim.x - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (!last || c + 1 >= m) return;
  __threadfence();
  gj_pivot_step(A, W, m, c + 1, fc, status);
}

void launch_gj_inverse(double* A, double* W, int m, double* fc, int* status, int* counter, cudaStream_t s) {
  const long long mm = (long long)m * m;
  const int nb = (int)std::min<long long>((mm + 255) / 256, 152 * 8);
  SD_COUNT(2 + m);
  launch_k(k_gj_init, dim3(nb), dim3(256), 0, s, W, m, status, counter);
  launch_k(k_gj_pivot, dim3(1), dim3(1024), 0, s, A, W, m, 0, fc, status);
  for (int c = 0; c < m; ++c) launch_k(k_gj_eliminate, dim3(nb), dim3(256), 0, s, A, W, m, c, fc, status, counter);
}

__global__ void k_identity_batch(double* X, long long stride, const int* idx, int m) {
  griddep_wait();
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m) X[(long long)k * stride + idx[k]] = 1.0;
}
void launch_identity_batch(double* X, long long stride, const int* idx, int m, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_identity_batch, dim3((m + 127) / 128), dim3(128), 0, s, X, stride, idx, m);
}

// A[r][k] = Y[k * stride + idx[r]]  (column k = operator applied to unit vector k)
__global__ void k_gather_dense(const double* Y, long long stride, const int* idx, int m, double* A) {
  griddep_wait();
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int r = (int)(e / m), k = (int)(e % m);
  A[e] = Y[(long long)k * stride + idx[r]];
}
void launch_gather_dense(const double* Y, long long stride, const int* idx, int m, double* A, cudaStream_t s) {
  SD_COUNT(1);
  const long long tot = (long long)m * m;
  launch_k(k_gather_dense, dim3((int)((tot + 255) / 256)), dim3(256), 0, s, Y, stride, idx, m, A);
}

__global__ void k_fill(double* x, double v, long long len) {
  griddep_wait();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    x[e] = v;
}
void launch_fill(double* x, double v, long long len, cudaStream_t s) {
  SD_COUNT(1); launch_k(k_fill, dim3(reduce_blocks(len)), dim3(RT), 0, s, x, v, len); }

// deterministic pseudo-random fill in [-1, 1] (start vector of the power iteration)
__global__ void k_hash_fill(double* x, long long len, unsigned seed) {
  griddep_wait();
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)e * 0x9E3779B97F4A7C15ull + seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}
void launch_hash_fill(double* x, long long len, unsigned seed, cudaStream_t s) {
  SD_COUNT(1);
  launch_k(k_hash_fill, dim3(reduce_blocks(len)), dim3(RT), 0, s, x, len, seed);
}

template void launch_dense_solve<float>(const double*, const int*, int, const float*, float*, cudaStream_t);
template void launch_dense_solve<double>(const double*, const int*, int, const double*, double*, cudaStream_t);

}  // namespace sdk
