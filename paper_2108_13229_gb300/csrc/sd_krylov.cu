// sd_krylov.cu -- FP64 kernels of the flexible GMRES(m) outer solve (the
// Krylov solver that replaces the paper's PD-GMRES, Sec. 5) and the dense
// coarsest-level solve of the multigrid V-cycles.
//
//  * multi-dot and fused update+dot kernels for classical Gram-Schmidt with
//    one re-orthogonalisation (CGS2): each block accumulates its slice of
//    all k dot products in registers, reduces them with warp shuffles and
//    writes one partial per block; a second kernel sums the partials in a
//    fixed order, so every reduction is deterministic (bitwise repeatable).
//  * Givens rotations, residual estimate and back substitution on the
//    (m+1) x m Hessenberg matrix, kept on the device (one thread).
//  * dense coarse solve x = A_c^{-1} b with the inverse built at setup by a
//    single-CTA Gauss-Jordan elimination with partial pivoting.
#include "sd_internal.cuh"

#include <math.h>

namespace sdk {

static const int RT = 256;      // threads per reduction block
static const int KMAX_REG = 32;  // max dot products per pass

int reduce_blocks(long long len) {
  long long nb = (len + RT * 4 - 1) / (RT * 4);
  if (nb > 152 * 4) nb = 152 * 4;
  if (nb < 1) nb = 1;
  return (int)nb;
}

// block-wide sum of acc[q] for q < k; result of q in partial[blockIdx.x*kmax+q]
__device__ __forceinline__ void block_sum_store(double* acc, int k, double* partial, int kmax) {
  __shared__ double sm[RT / 32][KMAX_REG];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < KMAX_REG; ++q) {
    if (q < k) {
      double v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) sm[warp][q] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < k) {
    double s = 0.0;
#pragma unroll
    for (int w = 0; w < RT / 32; ++w) s += sm[w][threadIdx.x];
    partial[(long long)blockIdx.x * kmax + threadIdx.x] = s;
  }
}

__global__ void __launch_bounds__(RT) k_mdot(const double* __restrict__ V, long long vs, int k,
                                             const double* __restrict__ w, long long len, double* __restrict__ partial,
                                             int kmax) {
  double acc[KMAX_REG];
#pragma unroll
  for (int q = 0; q < KMAX_REG; ++q) acc[q] = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < len; e += stride) {
    const double we = w[e];
#pragma unroll
    for (int q = 0; q < KMAX_REG; ++q)
      if (q < k) acc[q] = fma(V[q * vs + e], we, acc[q]);
  }
  block_sum_store(acc, k, partial, kmax);
}

void launch_mdot(const double* V, long long vstride, int k, const double* w, long long len, double* partial, int kmax,
                 int nblk, cudaStream_t s) {
  k_mdot<<<nblk, RT, 0, s>>>(V, vstride, k, w, len, partial, kmax);
}

// mode 1: w -= sum coef_q V_q, partial dots V_q . w   (second CGS pass)
// mode 2: w -= sum coef_q V_q, partial dot w . w      (norm of the new vector)
__global__ void __launch_bounds__(RT) k_mupdate(const double* __restrict__ V, long long vs, int k,
                                                const double* __restrict__ coef, double* __restrict__ w,
                                                long long len, double* __restrict__ partial, int kmax, int mode) {
  __shared__ double cf[KMAX_REG];
  if (threadIdx.x < KMAX_REG) cf[threadIdx.x] = threadIdx.x < k ? coef[threadIdx.x] : 0.0;
  __syncthreads();
  double acc[KMAX_REG];
#pragma unroll
  for (int q = 0; q < KMAX_REG; ++q) acc[q] = 0.0;
  const long long stride = (long long)gridDim.x * RT;
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < len; e += stride) {
    double we = w[e];
#pragma unroll
    for (int q = 0; q < KMAX_REG; ++q)
      if (q < k) we = fma(-cf[q], V[q * vs + e], we);
    w[e] = we;
    if (mode == 1) {
#pragma unroll
      for (int q = 0; q < KMAX_REG; ++q)
        if (q < k) acc[q] = fma(V[q * vs + e], we, acc[q]);
    } else {
      acc[0] = fma(we, we, acc[0]);
    }
  }
  block_sum_store(acc, mode == 1 ? k : 1, partial, kmax);
}

void launch_mupdate(const double* V, long long vstride, int k, const double* coef, double* w, long long len,
                    double* partial, int kmax, int nblk, int mode, cudaStream_t s) {
  k_mupdate<<<nblk, RT, 0, s>>>(V, vstride, k, coef, w, len, partial, kmax, mode);
}

__global__ void k_reduce(const double* __restrict__ partial, int nblk, int k, int kmax, double* __restrict__ out,
                         int accumulate) {
  // one warp per output; lanes sum strided partials, then a fixed shuffle tree
  const int q = blockIdx.x;
  if (q >= k) return;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += 32) s += partial[(long long)b * kmax + q];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (threadIdx.x == 0) out[q] = accumulate ? out[q] + s : s;
}

void launch_reduce(const double* partial, int nblk, int k, int kmax, double* out, int accumulate, cudaStream_t s) {
  k_reduce<<<k, 32, 0, s>>>(partial, nblk, k, kmax, out, accumulate);
}

void launch_dot(const double* a, const double* b, long long len, double* partial, int nblk, double* out,
                cudaStream_t s) {
  k_mdot<<<nblk, RT, 0, s>>>(a, 0, 1, b, len, partial, 1);
  k_reduce<<<1, 32, 0, s>>>(partial, nblk, 1, 1, out, 0);
}

// mode 0: y = sdev[0] * x ; mode 1: y = x / sqrt(sdev[0])
__global__ void k_scale_by(const double* __restrict__ x, double* __restrict__ y, long long len,
                           const double* __restrict__ sdev, int mode) {
  const double f = mode == 0 ? sdev[0] : 1.0 / sqrt(sdev[0]);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    y[e] = f * x[e];
}

void launch_scale_by(const double* x, double* y, long long len, const double* sdev, int mode, cudaStream_t s) {
  k_scale_by<<<reduce_blocks(len), RT, 0, s>>>(x, y, len, sdev, mode);
}

__global__ void __launch_bounds__(RT) k_axpy_multi(double* __restrict__ x, const double* __restrict__ Z, long long zs,
                                                   const double* __restrict__ y, int k, long long len) {
  __shared__ double cf[KMAX_REG];
  if (threadIdx.x < KMAX_REG) cf[threadIdx.x] = threadIdx.x < k ? y[threadIdx.x] : 0.0;
  __syncthreads();
  for (long long e = blockIdx.x * (long long)RT + threadIdx.x; e < len; e += (long long)gridDim.x * RT) {
    double xe = x[e];
#pragma unroll
    for (int q = 0; q < KMAX_REG; ++q)
      if (q < k) xe = fma(cf[q], Z[q * zs + e], xe);
    x[e] = xe;
  }
}

void launch_axpy_multi(double* x, const double* Z, long long zstride, const double* ycoef, int k, long long len,
                       cudaStream_t s) {
  k_axpy_multi<<<reduce_blocks(len), RT, 0, s>>>(x, Z, zstride, ycoef, k, len);
}

// ----------------------------------------------------- Hessenberg / Givens
// State layout (doubles): R[(m+1)*m] column-major (column j at j*(m+1)),
// cs[m], sn[m], g[m+1].  flag[0] = |g_{j+1}| (residual estimate),
// flag[1] = 1 / h_{j+1,j} (scale of the next basis vector), flag[2] = 1 on
// NaN/Inf, flag[3] = 1 on breakdown (h_{j+1,j} == 0).
__global__ void k_init_cycle(double* st, int m, const double* beta2, double* flag) {
  if (threadIdx.x != 0) return;
  double* g = st + (m + 1) * m + 2 * m;
  const double beta = sqrt(beta2[0]);
  g[0] = beta;
  for (int i = 1; i <= m; ++i) g[i] = 0.0;
  flag[0] = beta;
  flag[1] = beta > 0.0 ? 1.0 / beta : 0.0;
  flag[2] = isfinite(beta) ? 0.0 : 1.0;
  flag[3] = 0.0;
}

void launch_init_cycle(double* st, int m, const double* beta2, double* flag, cudaStream_t s) {
  k_init_cycle<<<1, 32, 0, s>>>(st, m, beta2, flag);
}

__global__ void k_givens(double* st, int j, int m, const double* h1, const double* h2, const double* nrm2,
                         double* flag) {
  if (threadIdx.x != 0) return;
  double* R = st;
  double* cs = st + (m + 1) * m;
  double* sn = cs + m;
  double* g = sn + m;
  double* col = R + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h1[i] + h2[i];
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
}

void launch_givens(double* st, int j, int m, const double* hcol1, const double* hcol2, const double* nrm2,
                   double* flag, cudaStream_t s) {
  k_givens<<<1, 32, 0, s>>>(st, j, m, hcol1, hcol2, nrm2, flag);
}

__global__ void k_backsolve(const double* st, int k, int m, double* y) {
  if (threadIdx.x != 0) return;
  const double* R = st;
  const double* g = st + (m + 1) * m + 2 * m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int l = i + 1; l < k; ++l) s -= R[(long long)l * (m + 1) + i] * y[l];
    y[i] = s / R[(long long)i * (m + 1) + i];
  }
}

void launch_backsolve(double* st, int k, int m, double* y, cudaStream_t s) { k_backsolve<<<1, 32, 0, s>>>(st, k, m, y); }

// ------------------------------------------------------ dense coarse solve
template <typename T>
__global__ void k_dense_solve(const double* __restrict__ Ainv, const int* __restrict__ idx, int m,
                              const T* __restrict__ b, T* __restrict__ x) {
  extern __shared__ double bs[];
  for (int l = threadIdx.x; l < m; l += blockDim.x) bs[l] = (double)b[idx[l]];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int r = warp; r < m; r += nw) {
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
  k_dense_solve<T><<<1, 512, sizeof(double) * m, s>>>(Ainv, idx, m, b, x);
}

// Gauss-Jordan with partial pivoting on [A | I], one CTA; the inverse ends in W.
__global__ void k_gj_inverse(double* A, double* W, int m, int* status) {
  extern __shared__ double fcol[];
  __shared__ int piv;
  __shared__ double pval;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (long long e = tid; e < (long long)m * m; e += nt) W[e] = ((e / m) == (e % m)) ? 1.0 : 0.0;
  if (tid == 0) *status = 0;
  __syncthreads();
  for (int c = 0; c < m; ++c) {
    if (tid == 0) {
      int p = c;
      double best = fabs(A[(long long)c * m + c]);
      for (int r = c + 1; r < m; ++r) {
        const double a = fabs(A[(long long)r * m + c]);
        if (a > best) { best = a; p = r; }
      }
      piv = p;
      pval = best;
      if (best == 0.0 && *status == 0) *status = c + 1;
    }
    __syncthreads();
    if (pval == 0.0) return;
    const int p = piv;
    if (p != c)
      for (int q = tid; q < m; q += nt) {
        double t = A[(long long)c * m + q]; A[(long long)c * m + q] = A[(long long)p * m + q]; A[(long long)p * m + q] = t;
        t = W[(long long)c * m + q]; W[(long long)c * m + q] = W[(long long)p * m + q]; W[(long long)p * m + q] = t;
      }
    __syncthreads();
    const double inv = 1.0 / A[(long long)c * m + c];
    __syncthreads();
    for (int q = tid; q < m; q += nt) {
      A[(long long)c * m + q] *= inv;
      W[(long long)c * m + q] *= inv;
    }
    __syncthreads();
    for (int r = tid; r < m; r += nt) fcol[r] = (r == c) ? 0.0 : A[(long long)r * m + c];
    __syncthreads();
    for (long long e = tid; e < (long long)m * m; e += nt) {
      const int r = (int)(e / m), q = (int)(e % m);
      const double f = fcol[r];
      if (f != 0.0) {
        A[e] -= f * A[(long long)c * m + q];
        W[e] -= f * W[(long long)c * m + q];
      }
    }
    __syncthreads();
  }
}

void launch_gj_inverse(double* A, double* work, int m, int* status, cudaStream_t s) {
  k_gj_inverse<<<1, 1024, sizeof(double) * m, s>>>(A, work, m, status);
}

__global__ void k_identity_batch(double* X, long long stride, const int* idx, int m) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < m) X[(long long)k * stride + idx[k]] = 1.0;
}
void launch_identity_batch(double* X, long long stride, const int* idx, int m, cudaStream_t s) {
  k_identity_batch<<<(m + 127) / 128, 128, 0, s>>>(X, stride, idx, m);
}

// A[r][k] = Y[k * stride + idx[r]]  (column k = operator applied to unit vector k)
__global__ void k_gather_dense(const double* Y, long long stride, const int* idx, int m, double* A) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)m * m) return;
  const int r = (int)(e / m), k = (int)(e % m);
  A[e] = Y[(long long)k * stride + idx[r]];
}
void launch_gather_dense(const double* Y, long long stride, const int* idx, int m, double* A, cudaStream_t s) {
  const long long tot = (long long)m * m;
  k_gather_dense<<<(int)((tot + 255) / 256), 256, 0, s>>>(Y, stride, idx, m, A);
}

__global__ void k_fill(double* x, double v, long long len) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x)
    x[e] = v;
}
void launch_fill(double* x, double v, long long len, cudaStream_t s) { k_fill<<<reduce_blocks(len), RT, 0, s>>>(x, v, len); }

// deterministic pseudo-random fill in [-1, 1] (start vector of the power iteration)
__global__ void k_hash_fill(double* x, long long len, unsigned seed) {
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = (unsigned long long)e * 0x9E3779B97F4A7C15ull + seed;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[e] = (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
  }
}
void launch_hash_fill(double* x, long long len, unsigned seed, cudaStream_t s) {
  k_hash_fill<<<reduce_blocks(len), RT, 0, s>>>(x, len, seed);
}

template void launch_dense_solve<float>(const double*, const int*, int, const float*, float*, cudaStream_t);
template void launch_dense_solve<double>(const double*, const int*, int, const double*, double*, cudaStream_t);

}  // namespace sdk
