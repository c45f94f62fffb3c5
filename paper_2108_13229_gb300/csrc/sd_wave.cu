// sd_wave.cu -- register-column smoothing of the fine FP32 multigrid levels
// (the V and D' blocks of the Sec. 4 block preconditioner, and the
// pressure-Laplacian block of its Schur approximation).
//
// NS Chebyshev steps in one kernel, as the shared-memory tiles of sd_ops.cu
// do, with the tile held in registers instead: each warp owns 32 columns
// (faces or cells) of TY output rows plus NS halo rows above and below, every
// lane its whole column.  A step computes all rows of the shrinking region
// at once (the rows are independent, so the lane has that much instruction-
// level parallelism); the vertical neighbours are the lane's own registers
// and the lateral ones come from the adjacent lanes by warp shuffles.  No
// shared memory, no block synchronisation and no index division remain in
// the step loops.  Each step loses one column per side (the edge lanes'
// outer neighbours are not in the warp), so a strip yields 32 - 2 NS output
// columns.  Per point the arithmetic is that of the per-step kernels (the
// value forms of sd_rows.cuh, in the same order), so the result is bitwise
// that of NS per-step launches.  Warps whose strip has no boundary column
// take the interior rows without their boundary masks.
#include "sd_internal.cuh"
#include "sd_rows.cuh"

namespace sdk {

namespace {

const unsigned kFull = 0xffffffffu;
const int kWarps = 4;  // warps (independent strips) per block

// One warp's tile of the velocity block.  IN: every row the steps compute
// (rows j0+1 .. j0+R-2) and every lane is an interior point of both the u and
// v rows, so the rows take no boundary case, no load is range checked and the
// right-hand side is held in registers; the code stays small enough for the
// instruction cache.  Otherwise each row takes its boundary cases.
template <int NS, int TY, bool IN>
__device__ __forceinline__ void col_tile_V(const Coef<float>& c, const float* __restrict__ xin,
                                           const float* __restrict__ b, float* __restrict__ xout,
                                           const ChebSteps<float>& cs, const float* __restrict__ ec, int nc, int Pc,
                                           int i, int j0, int lane) {
  constexpr int R = TY + 2 * NS;
  const int n = c.n, P = c.P;
  const long long nv = (long long)n * P;
  const bool ucol = i >= 0 && i <= n, vcol = i >= 0 && i < n;
  const float* ecu = ec;
  const float* ecv = ec ? ec + (long long)nc * Pc : nullptr;
  // the lane's column over rows j0 .. j0 + R - 1: iterate, d of the last step,
  // and (IN) the right-hand side
  float U[R], V[R], DU[R], DV[R], BU[IN ? R : 1], BV[IN ? R : 1];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = j0 + q;
    const long long k = (long long)j * P + i;
    float xu = 0.f, xv = 0.f;
    if (xin) {
      if (IN || (ucol && j >= 0 && j < n)) {
        xu = xin[k];
        if (ec && (IN || c.lat || (i > 0 && i < n))) xu += prolong_u_val(ecu, nc, nc, 0, Pc, i, j, c.lat);
      }
      if (IN || (vcol && j >= 0 && j <= n)) {
        xv = xin[nv + k];
        if (ec && (IN || j < n)) xv += prolong_v_val(ecv, nc, nc, 0, Pc, i, j);
      }
    }
    U[q] = xu;
    V[q] = xv;
    DU[q] = DV[q] = 0.f;
    if constexpr (IN) {
      BU[q] = (q > 0 && q < R - 1) ? b[k] : 0.f;
      BV[q] = (q > 0 && q < R - 1) ? b[nv + k] : 0.f;
    }
  }
#pragma unroll
  for (int s = 1; s <= NS; ++s) {
    const bool rd = s > 1 || xin != nullptr;
    const float a = cs.a[s - 1], cc = cs.c[s - 1];
    float NU[R], NV[R];
    // rows s .. R-1-s are valid after step s; the lateral neighbours of row q
    // come from the adjacent lanes, and uES = u(i+1, q-1) is the previous
    // row's shuffle
    float uEp = __shfl_down_sync(kFull, U[s - 1], 1);
#pragma unroll
    for (int q = s; q < R - s; ++q) {
      const int r = j0 + q;
      const float uC = U[q], uN = U[q + 1], uS = U[q - 1];
      const float vC = V[q], vN = V[q + 1], vS = V[q - 1];
      const float uW = __shfl_up_sync(kFull, uC, 1);
      const float uE = __shfl_down_sync(kFull, uC, 1);
      const float vE = __shfl_down_sync(kFull, vC, 1);
      const float vW = __shfl_up_sync(kFull, vC, 1);
      const float vNW = __shfl_up_sync(kFull, vN, 1);
      const float vSW = vW, uES = uEp;
      uEp = uE;
      const float adu = a != 0.f ? a * DU[q] : 0.f;
      const float adv = a != 0.f ? a * DV[q] : 0.f;
      const float xcu = rd ? uC : 0.f, xcv = rd ? vC : 0.f;
      float nu = 0.f, nvv = 0.f, du = 0.f, dv = 0.f;
      if constexpr (IN) {
        float off, dg;
        u_row_vals<float, true>(c, i, r, rd, uW, uE, uN, uS, vN, vNW, vC, vSW, off, dg);
        cheb_point(BU[q], xcu, off, dg, adu, cc, du, nu);
        v_row_vals<float, true>(c, i, r, rd, vS, vN, vE, vSW, uE, uES, uC, uS, off, dg);
        cheb_point(BV[q], xcv, off, dg, adv, cc, dv, nvv);
      } else {
        const long long k = (long long)r * P + i;
        if (ucol && r >= 0 && r < n) {
          if ((i == 0 || i == n) && !c.lat) {
            nu = b[k];
          } else {
            float off, dg;
            if (i == 0 || i == n)
              ub_row_vals<float>(c, i, r, rd, i == 0 ? uE : uW, uN, uS, i == 0 ? vN : vNW, i == 0 ? vC : vSW, off,
                                 dg);
            else u_row_vals<float, false>(c, i, r, rd, uW, uE, uN, uS, vN, vNW, vC, vSW, off, dg);
            cheb_point(b[k], xcu, off, dg, adu, cc, du, nu);
          }
        }
        if (vcol && r >= 0 && r <= n) {
          if (r == n) {
            nvv = b[nv + k];
          } else {
            float off, dg;
            v_row_vals<float, false>(c, i, r, rd, vS, vN, vE, vSW, uE, uES, uC, uS, off, dg);
            cheb_point(b[nv + k], xcv, off, dg, adv, cc, dv, nvv);
          }
        }
      }
      NU[q] = nu;
      NV[q] = nvv;
      DU[q] = du;
      DV[q] = dv;
    }
#pragma unroll
    for (int q = s; q < R - s; ++q) {
      U[q] = NU[q];
      V[q] = NV[q];
    }
  }
  if (lane >= NS && lane < 32 - NS) {
#pragma unroll
    for (int q = NS; q < NS + TY; ++q) {
      const int r = j0 + q;
      const long long k = (long long)r * P + i;
      if (IN || (ucol && r < n)) xout[k] = U[q];
      if (IN || (vcol && r <= n)) xout[nv + k] = V[q];
    }
  }
}

template <int NS, int TY, bool BT>
__global__ void __launch_bounds__(32 * kWarps, 4) k_wave_V(Coef<float> c, const float* __restrict__ xin,
                                                           const float* __restrict__ b, float* __restrict__ xout,
                                                           ChebSteps<float> cs, const float* __restrict__ ct,
                                                           const float* __restrict__ ec, int nc, int Pc, Bat bt) {
  griddep_wait();
  if constexpr (BT) {
    long long o;
    if (!bat_enter(bt, o)) return;
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    xout = bsh(xout, o);
    ec = bsh(ec, o);
    if (ct) {
      const float* q = bsh(ct, o);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        cs.a[s] = q[s];
        cs.c[s] = q[8 + s];
      }
    }
  }
  constexpr int W = 32 - 2 * NS, R = TY + 2 * NS;
  const int n = c.n;
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (strip * W > n) return;  // the whole warp: u faces are columns 0..n
  const int i0 = strip * W - NS, i = i0 + lane;
  const int j0 = blockIdx.y * TY - NS;  // row of register q = 0
  // no lane within two columns of a side, no computed row on a boundary row
  const bool inner = i0 >= 2 && i0 + 31 <= n - 2 && j0 + 1 >= 1 && j0 + R - 2 <= n - 2;
  if (inner) col_tile_V<NS, TY, true>(c, xin, b, xout, cs, ec, nc, Pc, i, j0, lane);
  else col_tile_V<NS, TY, false>(c, xin, b, xout, cs, ec, nc, Pc, i, j0, lane);
}

// One warp's tile of a cell block (D' or the pressure Laplacian).  IN: every
// computed row and lane is an interior cell (no boundary face), so nothing is
// range checked and the right-hand side is held in registers.
template <int NS, int TY, bool IN>
__device__ __forceinline__ void col_tile_D(const Coef<float>& c, const float* __restrict__ xin,
                                           const float* __restrict__ b, float* __restrict__ xout,
                                           const ChebSteps<float>& cs, const float* __restrict__ ec, int nc, int Pc,
                                           int i, int j0, int lane) {
  constexpr int R = TY + 2 * NS;
  const int n = c.n, P = c.P;
  const bool col = i >= 0 && i < n;
  // the x-face transmissibility of column i is read for i = 0..n (the east
  // face of the last cell is lane i = n's west face)
  const bool tcol = i >= 0 && i <= n;
  float X[R], D[R], TW[R], TN[R + 1], B[IN ? R : 1];
#pragma unroll
  for (int q = 0; q < R; ++q) {
    const int j = j0 + q;
    const long long k = (long long)j * P + i;
    float x = 0.f;
    if (xin && (IN || (col && j >= 0 && j < n))) {
      x = xin[k];
      if (ec) x += prolong_D_val(ec, nc, nc, Pc, i, j);
    }
    X[q] = x;
    D[q] = 0.f;
    // Tx(i, j) (west face); TN[q] = Ty(i, j) (the face below row j)
    TW[q] = (IN || (tcol && j >= 0 && j < n)) ? c.Tx[k] : 0.f;
    TN[q] = (IN || (col && j >= 0 && j <= n)) ? c.Ty[k] : 0.f;
    if constexpr (IN) B[q] = (q > 0 && q < R - 1) ? b[k] : 0.f;
  }
  {
    const int j = j0 + R;
    TN[R] = (IN || (col && j >= 0 && j <= n)) ? c.Ty[(long long)j * P + i] : 0.f;
  }
#pragma unroll
  for (int s = 1; s <= NS; ++s) {
    const bool rd = s > 1 || xin != nullptr;
    const float a = cs.a[s - 1], cc = cs.c[s - 1];
    float NX[R];
#pragma unroll
    for (int q = s; q < R - s; ++q) {
      const int r = j0 + q;
      const float pC = X[q], pN = X[q + 1], pS = X[q - 1];
      const float pW = __shfl_up_sync(kFull, pC, 1);
      const float pE = __shfl_down_sync(kFull, pC, 1);
      const float tw = TW[q], te = __shfl_down_sync(kFull, tw, 1), ts = TN[q], tn = TN[q + 1];
      const float ad = a != 0.f ? a * D[q] : 0.f;
      const float xc = rd ? pC : 0.f;
      float nx = 0.f, d = 0.f;
      if constexpr (IN) {
        float off, dg;
        d_row_vals<float, true>(c, i, r, rd, tw, te, ts, tn, pW, pE, pS, pN, off, dg);
        cheb_point(B[q], xc, off, dg, ad, cc, d, nx);
      } else if (col && r >= 0 && r < n) {
        float off, dg;
        d_row_vals<float, false>(c, i, r, rd, tw, te, ts, tn, pW, pE, pS, pN, off, dg);
        cheb_point(b[(long long)r * P + i], xc, off, dg, ad, cc, d, nx);
      }
      NX[q] = nx;
      D[q] = d;
    }
#pragma unroll
    for (int q = s; q < R - s; ++q) X[q] = NX[q];
  }
  if (lane >= NS && lane < 32 - NS && (IN || col)) {
#pragma unroll
    for (int q = NS; q < NS + TY; ++q) {
      const int r = j0 + q;
      if (IN || r < n) xout[(long long)r * P + i] = X[q];
    }
  }
}

template <int NS, int TY, bool BT>
__global__ void __launch_bounds__(32 * kWarps, 4) k_wave_D(Coef<float> c, const float* __restrict__ xin,
                                                           const float* __restrict__ b, float* __restrict__ xout,
                                                           ChebSteps<float> cs, const float* __restrict__ ct,
                                                           const float* __restrict__ ec, int nc, int Pc, Bat bt) {
  griddep_wait();
  if constexpr (BT) {
    long long o;
    if (!bat_enter(bt, o)) return;
    bsh_coef(c, o);
    xin = bsh(xin, o);
    b = bsh(b, o);
    xout = bsh(xout, o);
    ec = bsh(ec, o);
    if (ct) {
      const float* q = bsh(ct, o);
#pragma unroll
      for (int s = 0; s < NS; ++s) {
        cs.a[s] = q[s];
        cs.c[s] = q[8 + s];
      }
    }
  }
  constexpr int W = 32 - 2 * NS, R = TY + 2 * NS;
  const int n = c.n;
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * kWarps + (threadIdx.x >> 5);
  if (strip * W >= n) return;  // the whole warp: cells are columns 0..n-1
  const int i0 = strip * W - NS, i = i0 + lane;
  const int j0 = blockIdx.y * TY - NS;
  // every lane an interior cell column, every computed row an interior row
  // (the loaded rows j0 .. j0+R-1 and the face row j0+R are then in range)
  const bool inner = i0 >= 1 && i0 + 31 <= n - 2 && j0 + 1 >= 1 && j0 + R - 2 <= n - 2;
  if (inner) col_tile_D<NS, TY, true>(c, xin, b, xout, cs, ec, nc, Pc, i, j0, lane);
  else col_tile_D<NS, TY, false>(c, xin, b, xout, cs, ec, nc, Pc, i, j0, lane);
}

template <int NS, int TY>
void wave_V_ns(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
               const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  constexpr int W = 32 - 2 * NS;
  const int strips = (c.n + 1 + W - 1) / W;
  const dim3 g((strips + kWarps - 1) / kWarps, (c.n + 1 + TY - 1) / TY);
  if (t_bat.off) launch_k(k_wave_V<NS, TY, true>, g, dim3(32 * kWarps), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc);
  else launch_k(k_wave_V<NS, TY, false>, g, dim3(32 * kWarps), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc);
}

template <int NS, int TY>
void wave_D_ns(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
               const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  constexpr int W = 32 - 2 * NS;
  const int strips = (c.n + W - 1) / W;
  const dim3 g((strips + kWarps - 1) / kWarps, (c.n + TY - 1) / TY);
  if (t_bat.off) launch_k(k_wave_D<NS, TY, true>, g, dim3(32 * kWarps), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc);
  else launch_k(k_wave_D<NS, TY, false>, g, dim3(32 * kWarps), 0, s, c, x_in, b, x_out, cs, ct, ec, nc, Pc);
}

template <int TY>
int wave_V_hs(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
              const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  switch (cs.ns) {
    case 1: wave_V_ns<1, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 2: wave_V_ns<2, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 3: wave_V_ns<3, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 4: wave_V_ns<4, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    default: return -1;
  }
  return 0;
}

template <int TY>
int wave_D_hs(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
              const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  switch (cs.ns) {
    case 1: wave_D_ns<1, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 2: wave_D_ns<2, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 3: wave_D_ns<3, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 4: wave_D_ns<4, TY>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    default: return -1;
  }
  return 0;
}

}  // namespace

int launch_wave_V(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
                  const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  int rc;
  switch (cs.wave) {
    case 4: rc = wave_V_hs<4>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 8: rc = wave_V_hs<8>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    default: rc = -1;
  }
  if (rc == 0) SD_COUNT(1);
  return rc;
}

int launch_wave_D(const Coef<float>& c, const float* x_in, const float* b, float* x_out, const ChebSteps<float>& cs,
                  const float* ct, const float* ec, int nc, int Pc, cudaStream_t s) {
  int rc;
  switch (cs.wave) {
    case 4: rc = wave_D_hs<4>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    case 8: rc = wave_D_hs<8>(c, x_in, b, x_out, cs, ct, ec, nc, Pc, s); break;
    default: rc = -1;
  }
  if (rc == 0) SD_COUNT(1);
  return rc;
}

}  // namespace sdk
