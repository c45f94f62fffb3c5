// sd_rows.cuh -- the discrete rows of the velocity block V and the Darcy
// block D' (Sec. 2 discretisation, Eqs. (1)-(7)) and the grid-transfer
// values of their multigrid, shared by every stencil kernel of the library.
//
// Each row exists in two forms: a value form that takes the neighbour values
// already loaded (registers, shared memory, warp shuffles) and a pointer form
// that loads them from a padded array and calls the value form.  All
// smoothers -- one Chebyshev step per launch, the shared-memory tiles and the
// register wavefronts -- therefore perform the same operations in the same
// order at every point, and their results agree bit for bit.
#pragma once
#include "sd_internal.cuh"

namespace sdk {

// Jacobi-scaled update term r / diag of the smoothers: the fast FP32
// division in the FP32 hierarchy (a smoother needs no correctly rounded
// quotient), the IEEE division in FP64
__device__ __forceinline__ float sdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sdiv(double a, double b) { return a / b; }

// ------------------------------------------------------------------ rows
// A row masks the terms that do not exist at a boundary with selects and
// accumulates the others in a fixed order.  The value forms take, for a
// boundary point, the values the pointer forms load from clamped in-range
// addresses; those values only enter masked terms.
//
// Off-diagonal part and diagonal of the velocity-block row of interior u face
// (i, j), from uW = u(i-1,j), uE = u(i+1,j), uN = u(i,j+1), uS = u(i,j-1),
// vN = v(i,j+1), vNW = v(i-1,j+1), vS = v(i,j), vSW = v(i-1,j).
// IN: the caller guarantees 2 <= i <= n-2 and 1 <= j <= n-2 (no boundary term
// applies); the same operations in the same order, without the masks.
// floor face i (v face of row 0) lies on the interface
template <typename T>
__device__ __forceinline__ bool on_gamma(const Coef<T>& c, int i) {
  return i >= c.iw && i < c.iw + c.n;
}

template <typename T, bool IN = false>
__device__ __forceinline__ void u_row_vals(const Coef<T>& c, int i, int j, bool read, T uW, T uE, T uN, T uS, T vN,
                                           T vNW, T vS, T vSW, T& off, T& diag) {
  const int n = c.n, nx = c.nx;
  const T mu = c.mu;
  const bool top = !IN && j == n - 1, bot = !IN && j == 0;
  // the floor below: Gamma (BJS slip) over faces iw .. iw + n, else the wall
  const bool slip = bot && i >= c.iw && i <= c.iw + n;
  T dg = c.d6;  // interior: h^2/dt + 4 mu (normal stress) + mu + mu (shear)
  T wh = T(0);
  if (top) dg += mu;  // wall at half distance above: 2 mu instead of mu
  if (slip) {         // Gamma below: BJS shear instead of mu
    wh = c.w[i] * c.h;
    dg += T(2) * wh - mu;
  } else if (bot) {   // channel floor beside Gamma at half distance
    dg += mu;
  }
  diag = dg;
  if (!read) {
    off = T(0);
    return;
  }
  const T cW = (IN || c.lat || i - 1 >= 1) ? c.m2 : T(0), cE = (IN || c.lat || i + 1 <= nx - 1) ? c.m2 : T(0);
  T of = cW * uW;
  of = fma(cE, uE, of);
  if (!top) {
    of = fma(c.m1, uN, of);
    of = fma(c.m1, vN, of);
    of = fma(mu, vNW, of);
  }
  if (!bot) {
    of = fma(c.m1, uS, of);
    of = fma(mu, vS, of);
    of = fma(c.m1, vSW, of);
  } else if (slip) {
    // a floor face beside Gamma (at the interface's ends) is data
    of = fma(wh, (on_gamma(c, i) ? vS : T(0)) - (on_gamma(c, i - 1) ? vSW : T(0)), of);
  }
  off = of;
}

template <typename T, bool IN = false>
__device__ __forceinline__ void u_row(const Coef<T>& c, const T* __restrict__ u, const T* __restrict__ v, int i,
                                      int j, bool read, T& off, T& diag) {
  const int n = c.n, P = c.P;
  const bool top = !IN && j == n - 1, bot = !IN && j == 0;
  T uW = T(0), uE = T(0), uN = T(0), uS = T(0), vN = T(0), vNW = T(0), vS = T(0), vSW = T(0);
  if (read) {
    const int r0 = j * P, rN = (top ? j : j + 1) * P, rS = (bot ? j : j - 1) * P;
    const int rv1 = (j + 1) * P;
    uW = u[r0 + i - 1];
    uE = u[r0 + i + 1];
    uN = u[rN + i];
    uS = u[rS + i];
    vN = v[rv1 + i];
    vNW = v[rv1 + i - 1];
    vS = v[r0 + i];
    vSW = v[r0 + i - 1];
  }
  u_row_vals<T, IN>(c, i, j, read, uW, uE, uN, uS, vN, vNW, vS, vSW, off, diag);
}

// Same for the v face (i, j), 0 <= j <= n-1 (j = 0: interface half control
// volume), from vS = v(i,j-1), vN = v(i,j+1), vE = v(i+1,j), vW = v(i-1,j),
// uE = u(i+1,j), uES = u(i+1,j-1), uW = u(i,j), uWS = u(i,j-1).  At j = 0 the
// interface row reads vN, vE, vW, uE and uW only.
// IN: 1 <= i <= n-2 and 1 <= j <= n-2.
template <typename T, bool IN = false>
__device__ __forceinline__ void v_row_vals(const Coef<T>& c, int i, int j, bool read, T vS, T vN, T vE, T vW, T uE,
                                           T uES, T uW, T uWS, T& off, T& diag) {
  const int n = c.n, nx = c.nx;
  const T mu = c.mu, h = c.h;
  const bool left = !IN && i == 0, right = !IN && i == nx - 1;
  if (!IN && j == 0) {  // v_Gamma (the caller takes a floor face beside Gamma as Dirichlet)
    // corners: BJS (interior, or a traction side's corner at half distance)
    // or a Dirichlet side at half distance; at an end of Gamma inside the
    // channel the floor face beside it is data
    const T wl = (left && !c.lat) ? T(0) : c.w[i], wr = (right && !c.lat) ? T(0) : c.w[i + 1];
    const bool gl = on_gamma(c, i - 1), gr = on_gamma(c, i + 1);
    T dg = T(0.5) * c.cm + T(2) * mu + c.rg[i];
    dg += left ? (c.lat ? h * wl : mu) : T(0.5) * h * wl;
    dg += right ? (c.lat ? h * wr : mu) : T(0.5) * h * wr;
    diag = dg;
    if (!read) {
      off = T(0);
      return;
    }
    T of = c.m2 * vN;
    if (!left) {
      of = fma(wl * h, uW, of);
      if (gl) of = fma(T(-0.5) * h * wl, vW, of);
    } else if (c.lat) {
      of = fma(wl * h, uW, of);
    }
    if (!right) {
      of = fma(-wr * h, uE, of);
      if (gr) of = fma(T(-0.5) * h * wr, vE, of);
    } else if (c.lat) {
      of = fma(-wr * h, uE, of);
    }
    off = of;
    return;
  }
  T dg = c.d6;
  if (right) dg += mu;
  if (left) dg += mu;
  diag = dg;
  if (!read) {
    off = T(0);
    return;
  }
  const T cN = (IN || j + 1 <= n - 1) ? c.m2 : T(0);
  // the face below is a floor face beside Gamma (data) only in row 1
  const T cS = (IN || j > 1 || on_gamma(c, i)) ? c.m2 : T(0);
  T of = cS * vS;
  of = fma(cN, vN, of);
  if (!right) {
    of = fma(c.m1, vE, of);
    of = fma(c.m1, uE, of);
    of = fma(mu, uES, of);
  } else if (c.lat) {  // traction side: its u faces are unknowns
    of = fma(c.m1, uE, of);
    of = fma(mu, uES, of);
  }
  if (!left) {
    of = fma(c.m1, vW, of);
    of = fma(mu, uW, of);
    of = fma(c.m1, uWS, of);
  } else if (c.lat) {
    of = fma(mu, uW, of);
    of = fma(c.m1, uWS, of);
  }
  off = of;
}

template <typename T, bool IN = false>
__device__ __forceinline__ void v_row(const Coef<T>& c, const T* __restrict__ u, const T* __restrict__ v, int i,
                                      int j, bool read, T& off, T& diag) {
  const int P = c.P;
  const bool left = !IN && i == 0, right = !IN && i == c.nx - 1;
  T vS = T(0), vN = T(0), vE = T(0), vW = T(0), uE = T(0), uES = T(0), uW = T(0), uWS = T(0);
  if (read) {
    if (!IN && j == 0) {
      vN = v[P + i];
      uW = u[i];
      uE = u[i + 1];
      vW = v[left ? i : i - 1];
      vE = v[right ? i : i + 1];
    } else {
      const int r0 = j * P, rm = (j - 1) * P, rp = (j + 1) * P;
      const int iE = right ? i : i + 1, iW = left ? i : i - 1;
      vS = v[rm + i];
      vN = v[rp + i];
      vE = v[r0 + iE];
      vW = v[r0 + iW];
      uE = u[r0 + i + 1];
      uES = u[rm + i + 1];
      uW = u[r0 + i];
      uWS = u[rm + i];
    }
  }
  v_row_vals<T, IN>(c, i, j, read, vS, vN, vE, vW, uE, uES, uW, uWS, off, diag);
}

// Side u face (i = 0 or n) of a traction side: x-momentum balance of the
// half control volume inside the domain (as v_Gamma for the interface):
// normal stress through the adjacent cell centre (the side's traction goes
// to the right-hand side), shear through its top and bottom at the side,
// from the side's tangential velocity at half distance, the wall above the
// top row at half distance, and at the interface corner the eliminated BJS
// slip of Eq. (6).  The pressure term is added by the caller.  Values: uI =
// u(ii,j) of the inner neighbour face (ii = 1 or n-1), uN = u(i,j+1), uS =
// u(i,j-1), vNc = v(ic,j+1), vSc = v(ic,j) of the adjacent cell column ic.
template <typename T>
__device__ __forceinline__ void ub_row_vals(const Coef<T>& c, int i, int j, bool read, T uI, T uN, T uS, T vNc,
                                            T vSc, T& off, T& diag) {
  const int n = c.n;
  const T mu = c.mu;
  const bool rt = i == c.nx, top = j == n - 1, bot = j == 0;
  // the side's floor corner: on Gamma (square geometry) the eliminated BJS
  // slip, in the channel the wall at half distance
  const bool slip = bot && i >= c.iw && i <= c.iw + n;
  const T wh = slip ? c.w[i] * c.h : T(0);
  T dg = T(0.5) * c.cm + T(2) * mu;
  dg += top ? mu : T(0.5) * mu;
  dg += slip ? wh : (bot ? mu : T(0.5) * mu);
  diag = dg;
  if (!read) {
    off = T(0);
    return;
  }
  const T sg = rt ? T(-1) : T(1);
  T of = c.m2 * uI;
  if (!top) {
    of = fma(T(-0.5) * mu, uN, of);
    of = fma(-sg * mu, vNc, of);
  }
  if (!bot) {
    of = fma(T(-0.5) * mu, uS, of);
    of = fma(sg * mu, vSc, of);
  } else if (slip) {
    of = fma(sg * wh, vSc, of);
  }
  off = of;
}

template <typename T>
__device__ __forceinline__ void ub_row(const Coef<T>& c, const T* __restrict__ u, const T* __restrict__ v, int i,
                                       int j, bool read, T& off, T& diag) {
  const int n = c.n, nx = c.nx, P = c.P;
  const bool rt = i == nx, top = j == n - 1, bot = j == 0;
  T uI = T(0), uN = T(0), uS = T(0), vNc = T(0), vSc = T(0);
  if (read) {
    const int r0 = j * P;
    const int ii = rt ? nx - 1 : 1, ic = rt ? nx - 1 : 0;
    uI = u[r0 + ii];
    if (!top) {
      uN = u[r0 + P + i];
      vNc = v[r0 + P + ic];
    }
    if (!bot) uS = u[r0 - P + i];
    vSc = v[r0 + ic];
  }
  ub_row_vals<T>(c, i, j, read, uI, uN, uS, vNc, vSc, off, diag);
}

// Row of cell (i, j) of a cell block (Darcy D' without the interface flux,
// or the pressure Laplacian), 0 <= i < c.cx, from the transmissibilities of
// its faces (tw, te, ts, tn) and the neighbour values.
// IN: 1 <= i <= cx-2 and 1 <= j <= n-2.
template <typename T, bool IN = false>
__device__ __forceinline__ void d_row_vals(const Coef<T>& c, int i, int j, bool read, T tw, T te, T ts, T tn, T pW,
                                           T pE, T pS, T pN, T& off, T& diag) {
  const int n = c.n;
  diag = (tw + te) + (ts + tn);
  if (!read) {
    off = T(0);
    return;
  }
  const T cW = (IN || i > 0) ? tw : T(0), cE = (IN || i < c.cx - 1) ? te : T(0);
  const T cS = (IN || j > 0) ? ts : T(0), cN = (IN || j < n - 1) ? tn : T(0);
  T of = cW * pW;
  of = fma(cE, pE, of);
  of = fma(cS, pS, of);
  of = fma(cN, pN, of);
  off = -of;
}

template <typename T, bool IN = false>
__device__ __forceinline__ void d_row(const Coef<T>& c, const T* __restrict__ p, int i, int j, bool read, T& off,
                                      T& diag) {
  const int n = c.n, P = c.P;
  const int r0 = j * P;
  const T tw = c.Tx[r0 + i], te = c.Tx[r0 + i + 1];
  const T ts = c.Ty[r0 + i], tn = c.Ty[r0 + P + i];
  T pW = T(0), pE = T(0), pS = T(0), pN = T(0);
  if (read) {
    pW = p[r0 + ((IN || i > 0) ? i - 1 : i)];
    pE = p[r0 + ((IN || i < c.cx - 1) ? i + 1 : i)];
    pS = p[((IN || j > 0) ? r0 - P : r0) + i];
    pN = p[((IN || j < n - 1) ? r0 + P : r0) + i];
  }
  d_row_vals<T, IN>(c, i, j, read, tw, te, ts, tn, pW, pE, pS, pN, off, diag);
}

// One Chebyshev step at a point: r = b - (diag x + off), d = ad + c r / diag
// with ad = a d_prev (0 on a first step), x_new = x + d.
template <typename T>
__device__ __forceinline__ void cheb_point(T bk, T xc, T off, T dg, T ad, T cc, T& dn, T& xn) {
  const T r = bk - (dg * xc + off);
  dn = ad + sdiv(cc * r, dg);
  xn = xc + dn;
}

// ------------------------------------------------------------ transfers
// Prolongation of the velocity block is bilinear on the staggered grid:
//  u: linear in x between coarse faces (Dirichlet faces carry 0), cell-centred
//     in y with weights 3/4, 1/4; below coarse row 0 (the interface) the
//     ghost equals row 0, above the top row (wall) it is the negative.
//  v: linear in y between coarse faces (the Dirichlet top carries 0),
//     cell-centred in x with weights 3/4, 1/4 and negative ghosts at the walls.
// Restriction is its transpose applied to the fine residual.
// The coarse level has nc rows, nxc free-flow cells across and its interface
// under floor faces iwc .. iwc + nc - 1 (square geometry: nxc = nc, iwc = 0).
// In the channel the floor beside the interface is a wall: there the u ghost
// below row 0 is the negative of row 0 (as at the lid) and the floor v faces,
// Dirichlet, carry 0.
template <typename T>
__device__ __forceinline__ T cu_at(const T* eu, int nc, int nxc, int iwc, int Pc, int I, int J, int lat) {
  // coarse u with zero Dirichlet faces (traction sides: the side faces' own
  // values) and the y ghosts described above
  if (!lat && (I <= 0 || I >= nxc)) return T(0);
  if (J < 0) {
    const T e0 = eu[I];
    return (I >= iwc && I <= iwc + nc) ? e0 : -e0;
  }
  if (J > nc - 1) return -eu[(long long)(nc - 1) * Pc + I];
  return eu[(long long)J * Pc + I];
}
template <typename T>
__device__ __forceinline__ T cv_at(const T* ev, int nc, int nxc, int iwc, int Pc, int I, int J) {
  if (J >= nc) return T(0);
  if (J == 0 && iwc > 0 && (I < iwc || I >= iwc + nc)) return T(0);
  if (I < 0) return -ev[(long long)J * Pc];
  if (I > nxc - 1) return -ev[(long long)J * Pc + nxc - 1];
  return ev[(long long)J * Pc + I];
}

// increment of fine u face (i, j), 0 < i < 2 nxc, j < 2 nc
template <typename T>
__device__ __forceinline__ T prolong_u_val(const T* __restrict__ eu, int nc, int nxc, int iwc, int Pc, int i, int j,
                                           int lat = 0) {
  const int J = j >> 1, Jn = (j & 1) ? J + 1 : J - 1;
  T cy0, cy1;
  if (i & 1) {
    const int I = i >> 1;
    cy0 = T(0.5) * (cu_at(eu, nc, nxc, iwc, Pc, I, J, lat) + cu_at(eu, nc, nxc, iwc, Pc, I + 1, J, lat));
    cy1 = T(0.5) * (cu_at(eu, nc, nxc, iwc, Pc, I, Jn, lat) + cu_at(eu, nc, nxc, iwc, Pc, I + 1, Jn, lat));
  } else {
    const int I = i >> 1;
    cy0 = cu_at(eu, nc, nxc, iwc, Pc, I, J, lat);
    cy1 = cu_at(eu, nc, nxc, iwc, Pc, I, Jn, lat);
  }
  return T(0.75) * cy0 + T(0.25) * cy1;
}

// increment of fine v face (i, j), i < 2 nxc, j < 2 nc
template <typename T>
__device__ __forceinline__ T prolong_v_val(const T* __restrict__ ev, int nc, int nxc, int iwc, int Pc, int i, int j) {
  const int I = i >> 1, In = (i & 1) ? I + 1 : I - 1;
  T cx0, cx1;
  if (j & 1) {
    const int J = j >> 1;
    cx0 = T(0.5) * (cv_at(ev, nc, nxc, iwc, Pc, I, J) + cv_at(ev, nc, nxc, iwc, Pc, I, J + 1));
    cx1 = T(0.5) * (cv_at(ev, nc, nxc, iwc, Pc, In, J) + cv_at(ev, nc, nxc, iwc, Pc, In, J + 1));
  } else {
    const int J = j >> 1;
    cx0 = cv_at(ev, nc, nxc, iwc, Pc, I, J);
    cx1 = cv_at(ev, nc, nxc, iwc, Pc, In, J);
  }
  return T(0.75) * cx0 + T(0.25) * cx1;
}

// coarse cell block of nc rows and ncx cells across
template <typename T>
__device__ __forceinline__ T cd_at(const T* e, int nc, int ncx, int Pc, int I, int J) {
  // lateral sides and top of D' are no-flow (mirror), the bottom is Dirichlet (negative mirror)
  if (I < 0) I = 0;
  if (I > ncx - 1) I = ncx - 1;
  if (J < 0) return -e[I];
  if (J > nc - 1) J = nc - 1;
  return e[(long long)J * Pc + I];
}

template <typename T>
__device__ __forceinline__ T prolong_D_val(const T* __restrict__ e, int nc, int ncx, int Pc, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  const int In = (i & 1) ? I + 1 : I - 1, Jn = (j & 1) ? J + 1 : J - 1;
  return T(0.5625) * cd_at(e, nc, ncx, Pc, I, J) +
         T(0.1875) * (cd_at(e, nc, ncx, Pc, In, J) + cd_at(e, nc, ncx, Pc, I, Jn)) +
         T(0.0625) * cd_at(e, nc, ncx, Pc, In, Jn);
}

}  // namespace sdk
