/*
 * sd_oracle.c -- plain, slow FP64 CPU oracle for the time-dependent coupled
 * Stokes-Darcy system (arXiv 2108.13229, Sec. 2, Eqs. (1)-(9)).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is used by the tests, by the
 * smoke check and by the CPU-baseline leg of the benchmark.  The product
 * (the CUDA library) never links, loads or calls it, and it shares no code,
 * header or table with the CUDA path.
 *
 * What it computes: for every implicit-Euler step (Sec. 2, backward Euler in
 * time) it assembles the monolithic matrix A of Eq. (9) in CSR form, builds
 * the right-hand side b, and solves A x = b exactly (up to rounding) with a
 * banded LU factorisation with partial pivoting of its own.
 *
 * Discretisation (the paper names the schemes in Sec. 2 but prints no stencil;
 * this file implements the following reading of them):
 *   geometry     free flow  [0,1]x[1,2], porous medium [0,1]x[0,1],
 *                interface Gamma = {y = 1}, n x n cells each, h = 1/n.
 *   unknowns     u  on vertical ff faces   (n+1) x n, index j*(n+1)+i
 *                v  on horizontal ff faces n x (n+1), index j*n+i   (j=0: Gamma)
 *                p_ff at ff cell centres   n x n
 *                p_pm at pm cell centres   n x n
 *                DoF = 4n^2 + 2n (Table 1).
 *   Stokes       MAC staggered finite volumes, full symmetric stress
 *                tau = mu (grad v + grad v^T), rho = 1, every row integrated
 *                over its control volume (Eq. (1), (2)).
 *   Darcy        cell-centred TPFA, harmonic-mean transmissibilities
 *                (Eq. (3), (4)).
 *   coupling     Eq. (7): the Darcy cell below Gamma sees the flux h*v_Gamma;
 *                Eq. (5): the v_Gamma row is the momentum balance of the half
 *                control volume [1, 1+h/2] with the pm pressure on Gamma
 *                reconstructed by TPFA, p_Gamma = p_c - mu h/(2 K_c) v_Gamma;
 *                Eq. (6): Beavers-Joseph-Saffman, the slip velocity on Gamma
 *                is eliminated from the shear flux of the bottom u rows.
 *   time         backward Euler (Sec. 2), mass h^2/dt on velocity rows
 *                (h^2/(2 dt) on the half control volume of v_Gamma).
 *   boundaries   bc 0: the manufactured solution (below) gives Dirichlet
 *                velocity on the ff top, left and right sides, Dirichlet
 *                pressure on the pm bottom, no flow through the pm sides.
 *                Dirichlet velocity faces are kept as DoFs with identity rows;
 *                their values are moved into the right-hand side of every row
 *                that touches them.
 *                bc 1 and 2: the ff left and right sides are traction
 *                boundaries instead: the normal stress -p + 2 mu du/dx equals
 *                -P_b and the tangential velocity is V_b there.  The u faces
 *                on them are unknowns whose rows are the x-momentum balance of
 *                the half control volume inside the domain (as for v_Gamma),
 *                the corner shear taken at half distance from V_b and, at the
 *                interface corner, through the eliminated BJS slip.
 *                bc 1: P_b, V_b, top and pm data from the manufactured
 *                solution (a test of the traction rows).
 *                bc 2: the paper's pressure-driven problem (Sec. 5): P_b =
 *                p_in(t) = dp (1 - cos(pi min(t, t_end)/t_end))/2 on the left,
 *                0 on the right, V_b = 0, no slip on the top, p = 0 on the pm
 *                bottom, no flow through the pm sides, no sources.
 *
 * Manufactured solution (constructed for testing; the paper has none):
 *   psi = sin(pi x) phi(y),  phi(y) = 1 + A (y-1) + (y-1)^2,  A = pi^2 + 2,
 *   u = psi_y, v = -psi_x, p_ff = cos(pi x)(1 - 2 mu pi A),
 *   p_pm = cos(pi x) exp(pi (y-1)), all times (1+t).
 *   With mu = K = alpha_BJ = 1 it satisfies Eqs. (1)-(7) exactly, with the
 *   momentum forcing f = dv/dt - mu lap v + grad p and no Darcy source.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Manufactured solution                                                     */
/* ------------------------------------------------------------------------ */
static double mms_a(void) { return OR_PI * OR_PI + 2.0; }
static double mms_phi(double y) { double s = y - 1.0; return 1.0 + mms_a() * s + s * s; }
static double mms_dphi(double y) { return mms_a() + 2.0 * (y - 1.0); }

double or_mms_u(double x, double y, double t) { return sin(OR_PI * x) * mms_dphi(y) * (1.0 + t); }
double or_mms_v(double x, double y, double t) { return -OR_PI * cos(OR_PI * x) * mms_phi(y) * (1.0 + t); }
double or_mms_pff(double x, double y, double t, double mu) {
  (void)y;
  return cos(OR_PI * x) * (1.0 - 2.0 * mu * OR_PI * mms_a()) * (1.0 + t);
}
double or_mms_ppm(double x, double y, double t) { return cos(OR_PI * x) * exp(OR_PI * (y - 1.0)) * (1.0 + t); }
/* f = du/dt - mu lap u + dp/dx ; dv/dt - mu lap v + dp/dy (Eq. (1) with a source) */
double or_mms_fx(double x, double y, double t, double mu) {
  double s = 1.0 + t, sx = sin(OR_PI * x);
  return sx * mms_dphi(y) * (1.0 + mu * OR_PI * OR_PI * s)
         - OR_PI * (1.0 - 2.0 * mu * OR_PI * mms_a()) * sx * s;
}
double or_mms_fy(double x, double y, double t, double mu) {
  double s = 1.0 + t, cx = cos(OR_PI * x), ph = mms_phi(y);
  return -OR_PI * cx * ph - mu * OR_PI * cx * (OR_PI * OR_PI * ph - 2.0) * s;
}

/* ------------------------------------------------------------------------ */
/* Context                                                                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int n;
  int geo;                   /* 0: square free flow n x n; 1: channel 3n x n over the pm (see or_create_geo) */
  int nx, iw;                /* free-flow cells across (n or 3n), first free-flow column above the pm (0 or n) */
  double h, mu, alpha, dt;
  int bc;                    /* 0, 1, 2: see the header */
  double dp, tend;           /* bc 2: inflow pressure amplitude and ramp time */
  double *K;                 /* n*n, row j*n+i, j = 0 at y = 0 */
  int64_t ndof, nnz;
  int64_t *rowptr;
  int32_t *col;
  double *val;
  /* banded LU of the row/column permuted matrix */
  int32_t *perm;             /* perm[k] = original index at band position k */
  int32_t *iperm;            /* iperm[original] = band position */
  int kl, ku;
  int64_t ldab;
  double *ab;
  int32_t *ipiv;
  int factored;
} or_ctx;

static int64_t ix_u(int n, int i, int j) { return (int64_t)j * (n + 1) + i; }
static int64_t ix_v(int n, int i, int j) { return (int64_t)n * (n + 1) + (int64_t)j * n + i; }
static int64_t ix_pf(int n, int i, int j) { return 2 * (int64_t)n * (n + 1) + (int64_t)j * n + i; }
static int64_t ix_pm(int n, int i, int j) { return 2 * (int64_t)n * (n + 1) + (int64_t)n * n + (int64_t)j * n + i; }

int64_t or_dof_count(int n) { return 4 * (int64_t)n * n + 2 * (int64_t)n; }

static double kc(const or_ctx *c, int i, int j) { return c->K[(int64_t)j * c->n + i]; }
/* TPFA transmissibility between two pm cells: harmonic mean over mu (h/h = 1) */
static double t_harm(const or_ctx *c, double ka, double kb) { return 2.0 * ka * kb / (ka + kb) / c->mu; }
/* BJS shear coefficient mu/(h + 2 beta) at the interior interface u face i (1..n-1);
   beta = sqrt(K)/alpha with sqrt(K) the mean over the two pm cells below the face */
static double bjs_w(const or_ctx *c, int i) {
  int n = c->n;
  double sk = 0.5 * (sqrt(kc(c, i - 1, n - 1)) + sqrt(kc(c, i, n - 1)));
  double beta = sk / c->alpha;
  return c->mu / (c->h + 2.0 * beta);
}
/* BJS shear coefficient at a traction side's u face above Gamma (i = 0 or n):
   only one pm cell below it */
static double bjs_w_side(const or_ctx *c, int i) {
  int n = c->n, ic = i == 0 ? 0 : n - 1;
  double beta = sqrt(kc(c, ic, n - 1)) / c->alpha;
  return c->mu / (c->h + 2.0 * beta);
}
/* TPFA reconstruction of p_pm on Gamma adds mu h^2/(2 K_c) to the v_Gamma row */
static double gam_r(const or_ctx *c, int i) { return c->mu * c->h * c->h / (2.0 * kc(c, i, c->n - 1)); }

/* ------------------------------------------------------------------------ */
/* Row builder                                                               */
/* ------------------------------------------------------------------------ */
typedef struct { int64_t col[24]; double val[24]; int cnt; } row_t;
static void radd(row_t *r, int64_t col, double v) {
  for (int k = 0; k < r->cnt; ++k)
    if (r->col[k] == col) { r->val[k] += v; return; }
  r->col[r->cnt] = col; r->val[r->cnt] = v; r->cnt++;
}
static void rsort(row_t *r) {
  for (int a = 1; a < r->cnt; ++a) {
    int64_t cc = r->col[a]; double vv = r->val[a]; int b = a - 1;
    while (b >= 0 && r->col[b] > cc) { r->col[b + 1] = r->col[b]; r->val[b + 1] = r->val[b]; --b; }
    r->col[b + 1] = cc; r->val[b + 1] = vv;
  }
}

/* Build the row of DoF `row` (Eqs. (1)-(9) as integrated over its control volume). */
static void build_row(const or_ctx *c, int64_t row, row_t *r) {
  const int n = c->n;
  const double h = c->h, mu = c->mu, cm = h * h / c->dt;
  r->cnt = 0;
  const int64_t nu = (int64_t)n * (n + 1), nv = nu, np = (int64_t)n * n;
  const int lat = c->bc != 0;  /* traction sides */
  if (row < nu) { /* u row */
    int j = (int)(row / (n + 1)), i = (int)(row % (n + 1));
    if ((i == 0 || i == n) && !lat) { radd(r, row, 1.0); return; }
    if (i == 0 || i == n) {                      /* traction side: half control volume */
      const double sg = i == 0 ? 1.0 : -1.0;     /* mirror for the right side */
      const int ii = i == 0 ? 1 : n - 1;         /* inner u neighbour */
      const int ic = i == 0 ? 0 : n - 1;         /* adjacent ff cell column */
      double diag = 0.5 * cm + 2.0 * mu;
      radd(r, ix_u(n, ii, j), -2.0 * mu);
      radd(r, ix_pf(n, ic, j), sg * h);
      if (j < n - 1) {
        diag += 0.5 * mu;
        radd(r, ix_u(n, i, j + 1), -0.5 * mu);
        radd(r, ix_v(n, ic, j + 1), -sg * mu);
      } else {
        diag += mu;                              /* wall at y = 2, half distance */
      }
      if (j > 0) {
        diag += 0.5 * mu;
        radd(r, ix_u(n, i, j - 1), -0.5 * mu);
        radd(r, ix_v(n, ic, j), sg * mu);
      } else {                                   /* interface corner: BJS slip eliminated */
        double w = bjs_w_side(c, i);
        diag += h * w;
        radd(r, ix_v(n, ic, 0), sg * h * w);
      }
      radd(r, row, diag);
      return;
    }
    double diag = cm + 4.0 * mu;                 /* BE mass + normal stress 2mu d2u/dx2 */
    if (i - 1 >= 1 || lat) radd(r, ix_u(n, i - 1, j), -2.0 * mu);
    if (i + 1 <= n - 1 || lat) radd(r, ix_u(n, i + 1, j), -2.0 * mu);
    if (j < n - 1) {                             /* shear through the top corner */
      diag += mu;
      radd(r, ix_u(n, i, j + 1), -mu);
      radd(r, ix_v(n, i, j + 1), -mu);
      radd(r, ix_v(n, i - 1, j + 1), mu);
    } else {                                     /* wall at y = 2, half-cell distance */
      diag += 2.0 * mu;
    }
    if (j > 0) {                                 /* shear through the bottom corner */
      diag += mu;
      radd(r, ix_u(n, i, j - 1), -mu);
      radd(r, ix_v(n, i, j), mu);
      radd(r, ix_v(n, i - 1, j), -mu);
    } else {                                     /* Gamma: BJS slip eliminated, Eq. (6) */
      double w = bjs_w(c, i);
      diag += 2.0 * w * h;
      radd(r, ix_v(n, i, 0), w * h);
      radd(r, ix_v(n, i - 1, 0), -w * h);
    }
    radd(r, ix_pf(n, i, j), h);                  /* pressure gradient (block B) */
    radd(r, ix_pf(n, i - 1, j), -h);
    radd(r, row, diag);
    return;
  }
  row -= nu;
  if (row < nv) { /* v row */
    int j = (int)(row / n), i = (int)(row % n);
    int64_t me = ix_v(n, i, j);
    if (j == n) { radd(r, me, 1.0); return; }
    if (j == 0) {                                /* v_Gamma: half control volume, Eq. (5) */
      double diag = 0.5 * cm + 2.0 * mu + gam_r(c, i);
      if (n > 1) radd(r, ix_v(n, i, 1), -2.0 * mu);
      radd(r, ix_pf(n, i, 0), h);
      radd(r, ix_pm(n, i, n - 1), -h);           /* block B'_1 */
      if (i > 0) {
        double w = bjs_w(c, i);
        radd(r, ix_u(n, i, 0), w * h);
        radd(r, ix_v(n, i - 1, 0), -0.5 * h * w);
        diag += 0.5 * h * w;
      } else if (lat) {                          /* traction side corner, BJS */
        double w = bjs_w_side(c, 0);
        radd(r, ix_u(n, 0, 0), w * h);
        diag += h * w;
      } else {
        diag += mu;
      }
      if (i < n - 1) {
        double w = bjs_w(c, i + 1);
        radd(r, ix_u(n, i + 1, 0), -w * h);
        radd(r, ix_v(n, i + 1, 0), -0.5 * h * w);
        diag += 0.5 * h * w;
      } else if (lat) {
        double w = bjs_w_side(c, n);
        radd(r, ix_u(n, n, 0), -w * h);
        diag += h * w;
      } else {
        diag += mu;
      }
      radd(r, me, diag);
      return;
    }
    double diag = cm + 4.0 * mu;
    radd(r, ix_v(n, i, j - 1), -2.0 * mu);
    if (j + 1 <= n - 1) radd(r, ix_v(n, i, j + 1), -2.0 * mu);
    if (i < n - 1) {
      diag += mu;
      radd(r, ix_v(n, i + 1, j), -mu);
      radd(r, ix_u(n, i + 1, j), -mu);
      radd(r, ix_u(n, i + 1, j - 1), mu);
    } else {
      diag += 2.0 * mu;                          /* tangential velocity given at half distance */
      if (lat) {
        radd(r, ix_u(n, n, j), -mu);
        radd(r, ix_u(n, n, j - 1), mu);
      }
    }
    if (i > 0) {
      diag += mu;
      radd(r, ix_v(n, i - 1, j), -mu);
      radd(r, ix_u(n, i, j), mu);
      radd(r, ix_u(n, i, j - 1), -mu);
    } else {
      diag += 2.0 * mu;
      if (lat) {
        radd(r, ix_u(n, 0, j), mu);
        radd(r, ix_u(n, 0, j - 1), -mu);
      }
    }
    radd(r, ix_pf(n, i, j), h);
    radd(r, ix_pf(n, i, j - 1), -h);
    radd(r, me, diag);
    return;
  }
  row -= nv;
  if (row < np) { /* continuity of ff cell (i, j), Eq. (2) */
    int j = (int)(row / n), i = (int)(row % n);
    if (i + 1 <= n - 1 || lat) radd(r, ix_u(n, i + 1, j), h);
    if (i >= 1 || lat) radd(r, ix_u(n, i, j), -h);
    if (j + 1 <= n - 1) radd(r, ix_v(n, i, j + 1), h);
    radd(r, ix_v(n, i, j), -h);
    return;
  }
  row -= np;
  { /* Darcy cell (i, j), Eqs. (3), (4), (7) */
    int j = (int)(row / n), i = (int)(row % n);
    int64_t me = ix_pm(n, i, j);
    double diag = 0.0, t;
    if (i > 0) { t = t_harm(c, kc(c, i - 1, j), kc(c, i, j)); diag += t; radd(r, ix_pm(n, i - 1, j), -t); }
    if (i < n - 1) { t = t_harm(c, kc(c, i + 1, j), kc(c, i, j)); diag += t; radd(r, ix_pm(n, i + 1, j), -t); }
    if (j > 0) { t = t_harm(c, kc(c, i, j - 1), kc(c, i, j)); diag += t; radd(r, ix_pm(n, i, j - 1), -t); }
    else { diag += 2.0 * kc(c, i, j) / c->mu; }  /* Dirichlet pressure at y = 0 */
    if (j < n - 1) { t = t_harm(c, kc(c, i, j + 1), kc(c, i, j)); diag += t; radd(r, ix_pm(n, i, j + 1), -t); }
    else { radd(r, ix_v(n, i, 0), h); }         /* block C'_1: outflow h v_Gamma, Eq. (7) */
    radd(r, me, diag);
  }
}


/* ------------------------------------------------------------------------ */
/* Channel geometry (geo 1): the model problem's free flow of Sec. 5, a      */
/* channel three times as wide as the porous medium.  Free flow             */
/* [-1,2] x [1,2] (3n x n cells) over the porous medium [0,1] x [0,1]; the  */
/* interface Gamma is the middle third of the channel's floor (free-flow    */
/* columns iw .. iw+n-1, iw = n), the rest of the floor a wall.  Unknowns:   */
/* u (3n+1) x n, v 3n x (n+1) (row 0: floor faces; the ones on Gamma are    */
/* the interface unknowns, the others wall faces with identity rows),       */
/* p_ff 3n x n, p_pm n x n: 10 n^2 + 4 n.                                    */
/* Rows follow the square geometry's reading; what changes at the floor:    */
/*  - u faces above the wall take the wall shear at half distance (as the   */
/*    lid does);                                                            */
/*  - u faces above Gamma take the eliminated BJS slip of Eq. (6); at the   */
/*    two ends of Gamma (x = 0, 1) the slip uses the one pm cell below and  */
/*    the wall face beside it enters as data;                               */
/*  - the v_Gamma rows are the half control volumes of Eq. (5), their end   */
/*    corners through those end faces;                                      */
/*  - traction ends (bc 1, 2) at x = -1 and x = 2, their floor corner at    */
/*    half distance from the wall.                                          */
/* ------------------------------------------------------------------------ */
static int64_t chu(const or_ctx *c, int i, int j) { return (int64_t)j * (c->nx + 1) + i; }
static int64_t chv(const or_ctx *c, int i, int j) { return (int64_t)c->n * (c->nx + 1) + (int64_t)j * c->nx + i; }
static int64_t chp(const or_ctx *c, int i, int j) {
  return (int64_t)c->n * (c->nx + 1) + (int64_t)(c->n + 1) * c->nx + (int64_t)j * c->nx + i;
}
static int64_t chm(const or_ctx *c, int i, int j) {
  return (int64_t)c->n * (c->nx + 1) + (int64_t)(c->n + 1) * c->nx + (int64_t)c->n * c->nx + (int64_t)j * c->n + i;
}
int64_t or_dof_count_geo(int n, int geo) {
  return geo == 1 ? 10 * (int64_t)n * n + 4 * (int64_t)n : or_dof_count(n);
}
/* x of free-flow u face i (a cell's centre is h/2 further) */
static double chx(const or_ctx *c, int i) { return (i - c->iw) * c->h; }
/* floor face i (v face, row 0) lies on Gamma */
static int on_gamma(const or_ctx *c, int i) { return i >= c->iw && i < c->iw + c->n; }
/* BJS coefficient mu / (h + 2 beta) at the floor corner of u face i, iw <= i <= iw + n:
   beta = sqrt(K)/alpha with sqrt(K) the mean over the pm cells below that lie under Gamma */
static double bjs_w_ch(const or_ctx *c, int i) {
  const int n = c->n, p = i - c->iw;
  double sk;
  if (p == 0) sk = sqrt(kc(c, 0, n - 1));
  else if (p == n) sk = sqrt(kc(c, n - 1, n - 1));
  else sk = 0.5 * (sqrt(kc(c, p - 1, n - 1)) + sqrt(kc(c, p, n - 1)));
  return c->mu / (c->h + 2.0 * sk / c->alpha);
}

static void build_row_channel(const or_ctx *c, int64_t row, row_t *r) {
  const int n = c->n, NX = c->nx;
  const double h = c->h, mu = c->mu, cm = h * h / c->dt;
  const int lat = c->bc != 0;
  const int64_t nu = (int64_t)n * (NX + 1), nv = (int64_t)NX * (n + 1), np = (int64_t)NX * n;
  r->cnt = 0;
  if (row < nu) { /* u row */
    const int j = (int)(row / (NX + 1)), i = (int)(row % (NX + 1));
    if ((i == 0 || i == NX) && !lat) { radd(r, row, 1.0); return; }
    if (i == 0 || i == NX) {                     /* traction end: half control volume */
      const double sg = i == 0 ? 1.0 : -1.0;
      const int ii = i == 0 ? 1 : NX - 1, ic = i == 0 ? 0 : NX - 1;
      double diag = 0.5 * cm + 2.0 * mu;
      radd(r, chu(c, ii, j), -2.0 * mu);
      radd(r, chp(c, ic, j), sg * h);
      if (j < n - 1) {
        diag += 0.5 * mu;
        radd(r, chu(c, i, j + 1), -0.5 * mu);
        radd(r, chv(c, ic, j + 1), -sg * mu);
      } else {
        diag += mu;                              /* lid at half distance */
      }
      if (j > 0) {
        diag += 0.5 * mu;
        radd(r, chu(c, i, j - 1), -0.5 * mu);
        radd(r, chv(c, ic, j), sg * mu);
      } else {
        diag += mu;                              /* channel floor at half distance */
      }
      radd(r, row, diag);
      return;
    }
    double diag = cm + 4.0 * mu;
    if (i - 1 >= 1 || lat) radd(r, chu(c, i - 1, j), -2.0 * mu);
    if (i + 1 <= NX - 1 || lat) radd(r, chu(c, i + 1, j), -2.0 * mu);
    if (j < n - 1) {
      diag += mu;
      radd(r, chu(c, i, j + 1), -mu);
      radd(r, chv(c, i, j + 1), -mu);
      radd(r, chv(c, i - 1, j + 1), mu);
    } else {
      diag += 2.0 * mu;
    }
    if (j > 0) {
      diag += mu;
      radd(r, chu(c, i, j - 1), -mu);
      radd(r, chv(c, i, j), mu);
      radd(r, chv(c, i - 1, j), -mu);
    } else if (i >= c->iw && i <= c->iw + n) {   /* over Gamma: BJS slip eliminated, Eq. (6) */
      const double w = bjs_w_ch(c, i);
      diag += 2.0 * w * h;
      if (on_gamma(c, i)) radd(r, chv(c, i, 0), w * h);
      if (on_gamma(c, i - 1)) radd(r, chv(c, i - 1, 0), -w * h);
    } else {
      diag += 2.0 * mu;                          /* channel floor, half-cell distance */
    }
    radd(r, chp(c, i, j), h);
    radd(r, chp(c, i - 1, j), -h);
    radd(r, row, diag);
    return;
  }
  row -= nu;
  if (row < nv) { /* v row */
    const int j = (int)(row / NX), i = (int)(row % NX);
    const int64_t me = chv(c, i, j);
    if (j == n || (j == 0 && !on_gamma(c, i))) { radd(r, me, 1.0); return; }
    if (j == 0) {                                /* v_Gamma: half control volume, Eq. (5) */
      const int p = i - c->iw;
      double diag = 0.5 * cm + 2.0 * mu + mu * h * h / (2.0 * kc(c, p, n - 1));
      if (n > 1) radd(r, chv(c, i, 1), -2.0 * mu);
      radd(r, chp(c, i, 0), h);
      radd(r, chm(c, p, n - 1), -h);             /* block B'_1 */
      double w = bjs_w_ch(c, i);
      radd(r, chu(c, i, 0), w * h);
      if (on_gamma(c, i - 1)) radd(r, chv(c, i - 1, 0), -0.5 * h * w);
      diag += 0.5 * h * w;
      w = bjs_w_ch(c, i + 1);
      radd(r, chu(c, i + 1, 0), -w * h);
      if (on_gamma(c, i + 1)) radd(r, chv(c, i + 1, 0), -0.5 * h * w);
      diag += 0.5 * h * w;
      radd(r, me, diag);
      return;
    }
    double diag = cm + 4.0 * mu;
    if (j - 1 >= 1 || on_gamma(c, i)) radd(r, chv(c, i, j - 1), -2.0 * mu);
    if (j + 1 <= n - 1) radd(r, chv(c, i, j + 1), -2.0 * mu);
    if (i < NX - 1) {
      diag += mu;
      radd(r, chv(c, i + 1, j), -mu);
      radd(r, chu(c, i + 1, j), -mu);
      radd(r, chu(c, i + 1, j - 1), mu);
    } else {
      diag += 2.0 * mu;
      if (lat) {
        radd(r, chu(c, NX, j), -mu);
        radd(r, chu(c, NX, j - 1), mu);
      }
    }
    if (i > 0) {
      diag += mu;
      radd(r, chv(c, i - 1, j), -mu);
      radd(r, chu(c, i, j), mu);
      radd(r, chu(c, i, j - 1), -mu);
    } else {
      diag += 2.0 * mu;
      if (lat) {
        radd(r, chu(c, 0, j), mu);
        radd(r, chu(c, 0, j - 1), -mu);
      }
    }
    radd(r, chp(c, i, j), h);
    radd(r, chp(c, i, j - 1), -h);
    radd(r, me, diag);
    return;
  }
  row -= nv;
  if (row < np) { /* continuity of ff cell (i, j), Eq. (2) */
    const int j = (int)(row / NX), i = (int)(row % NX);
    if (i + 1 <= NX - 1 || lat) radd(r, chu(c, i + 1, j), h);
    if (i >= 1 || lat) radd(r, chu(c, i, j), -h);
    if (j + 1 <= n - 1) radd(r, chv(c, i, j + 1), h);
    if (j > 0 || on_gamma(c, i)) radd(r, chv(c, i, j), -h);
    return;
  }
  row -= np;
  { /* Darcy cell (i, j), Eqs. (3), (4), (7); the cells below Gamma are its columns iw .. iw+n-1 */
    const int j = (int)(row / n), i = (int)(row % n);
    const int64_t me = chm(c, i, j);
    double diag = 0.0, t;
    if (i > 0) { t = t_harm(c, kc(c, i - 1, j), kc(c, i, j)); diag += t; radd(r, chm(c, i - 1, j), -t); }
    if (i < n - 1) { t = t_harm(c, kc(c, i + 1, j), kc(c, i, j)); diag += t; radd(r, chm(c, i + 1, j), -t); }
    if (j > 0) { t = t_harm(c, kc(c, i, j - 1), kc(c, i, j)); diag += t; radd(r, chm(c, i, j - 1), -t); }
    else { diag += 2.0 * kc(c, i, j) / c->mu; }
    if (j < n - 1) { t = t_harm(c, kc(c, i, j + 1), kc(c, i, j)); diag += t; radd(r, chm(c, i, j + 1), -t); }
    else { radd(r, chv(c, c->iw + i, 0), h); }  /* block C'_1: outflow h v_Gamma, Eq. (7) */
    radd(r, me, diag);
  }
}

/* geo 0: the square free flow over the square porous medium (Table 1);
   geo 1: the channel above */
or_ctx *or_create_geo(int n, double mu, double alpha, double dt, const double *K, int bc, double dp, double tend,
                      int geo) {
  if (n < 2 || !(mu > 0) || !(alpha > 0) || !(dt > 0) || !K || bc < 0 || bc > 2 || !(tend > 0) || geo < 0 ||
      geo > 1)
    return NULL;
  or_ctx *c = (or_ctx *)calloc(1, sizeof(or_ctx));
  c->n = n; c->h = 1.0 / n; c->mu = mu; c->alpha = alpha; c->dt = dt;
  c->geo = geo; c->nx = geo == 1 ? 3 * n : n; c->iw = geo == 1 ? n : 0;
  c->bc = bc; c->dp = dp; c->tend = tend;
  c->K = (double *)malloc(sizeof(double) * (size_t)n * n);
  memcpy(c->K, K, sizeof(double) * (size_t)n * n);
  c->ndof = or_dof_count_geo(n, geo);
  c->rowptr = (int64_t *)malloc(sizeof(int64_t) * (size_t)(c->ndof + 1));
  int64_t cap = c->ndof * 12;
  c->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
  c->val = (double *)malloc(sizeof(double) * (size_t)cap);
  row_t r;
  int64_t nz = 0;
  c->rowptr[0] = 0;
  for (int64_t row = 0; row < c->ndof; ++row) {
    if (geo == 1) build_row_channel(c, row, &r);
    else build_row(c, row, &r);
    rsort(&r);
    for (int k = 0; k < r.cnt; ++k) { c->col[nz] = (int32_t)r.col[k]; c->val[nz] = r.val[k]; ++nz; }
    c->rowptr[row + 1] = nz;
  }
  c->nnz = nz;
  return c;
}

or_ctx *or_create_bc(int n, double mu, double alpha, double dt, const double *K, int bc, double dp, double tend) {
  return or_create_geo(n, mu, alpha, dt, K, bc, dp, tend, 0);
}

or_ctx *or_create(int n, double mu, double alpha, double dt, const double *K) {
  return or_create_bc(n, mu, alpha, dt, K, 0, 0.0, 1.0);
}

void or_destroy(or_ctx *c) {
  if (!c) return;
  free(c->K); free(c->rowptr); free(c->col); free(c->val);
  free(c->perm); free(c->iperm); free(c->ab); free(c->ipiv);
  free(c);
}

int64_t or_ndof(const or_ctx *c) { return c->ndof; }
int64_t or_nnz(const or_ctx *c) { return c->nnz; }
void or_get_csr(const or_ctx *c, int64_t *rowptr, int32_t *col, double *val) {
  memcpy(rowptr, c->rowptr, sizeof(int64_t) * (size_t)(c->ndof + 1));
  memcpy(col, c->col, sizeof(int32_t) * (size_t)c->nnz);
  memcpy(val, c->val, sizeof(double) * (size_t)c->nnz);
}

/* y = A x */
void or_apply(const or_ctx *c, const double *x, double *y) {
  for (int64_t r = 0; r < c->ndof; ++r) {
    double s = 0.0;
    for (int64_t k = c->rowptr[r]; k < c->rowptr[r + 1]; ++k) s += c->val[k] * x[c->col[k]];
    y[r] = s;
  }
}

/* ------------------------------------------------------------------------ */
/* Exact (manufactured) solution sampled at the DoF locations                */
/* ------------------------------------------------------------------------ */
void or_exact(int n, double t, double mu, double *x) {
  double h = 1.0 / n;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= n; ++i) x[ix_u(n, i, j)] = or_mms_u(i * h, 1.0 + (j + 0.5) * h, t);
  for (int j = 0; j <= n; ++j)
    for (int i = 0; i < n; ++i) x[ix_v(n, i, j)] = or_mms_v((i + 0.5) * h, 1.0 + j * h, t);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      x[ix_pf(n, i, j)] = or_mms_pff((i + 0.5) * h, 1.0 + (j + 0.5) * h, t, mu);
      x[ix_pm(n, i, j)] = or_mms_ppm((i + 0.5) * h, (j + 0.5) * h, t);
    }
}

/* ------------------------------------------------------------------------ */
/* Right-hand side of the implicit-Euler step to time t (Sec. 2)             */
/* xprev: solution at the previous time level (only its velocities enter)    */
/* ------------------------------------------------------------------------ */
/* inflow pressure of the paper's problem (bc 2): half cosine from 0 to dp over [0, t_end] */
double or_p_in(double dp, double tend, double t) {
  double s = t < tend ? t : tend;
  return dp * 0.5 * (1.0 - cos(OR_PI * s / tend));
}

/* traction-side data: P_b (minus the prescribed normal stress) and V_b (tangential velocity) */
static double side_p(const or_ctx *c, int right, double y, double t) {
  if (c->bc == 2) return right ? 0.0 : or_p_in(c->dp, c->tend, t);
  double x = right ? 1.0 : 0.0;
  double ux = OR_PI * cos(OR_PI * x) * mms_dphi(y) * (1.0 + t);  /* du/dx of the manufactured u */
  return or_mms_pff(x, y, t, c->mu) - 2.0 * c->mu * ux;
}
static double side_v(const or_ctx *c, int right, double y, double t) {
  return c->bc == 2 ? 0.0 : or_mms_v(right ? 1.0 : 0.0, y, t);
}
/* boundary data of the other sides and the sources: manufactured (bc 0, 1) or zero (bc 2) */
static double dat_u(const or_ctx *c, double x, double y, double t) { return c->bc == 2 ? 0.0 : or_mms_u(x, y, t); }
static double dat_v(const or_ctx *c, double x, double y, double t) { return c->bc == 2 ? 0.0 : or_mms_v(x, y, t); }
static double dat_ppm(const or_ctx *c, double x, double y, double t) { return c->bc == 2 ? 0.0 : or_mms_ppm(x, y, t); }
static double dat_fx(const or_ctx *c, double x, double y, double t) {
  return c->bc == 2 ? 0.0 : or_mms_fx(x, y, t, c->mu);
}
static double dat_fy(const or_ctx *c, double x, double y, double t) {
  return c->bc == 2 ? 0.0 : or_mms_fy(x, y, t, c->mu);
}

static void rhs_channel(const or_ctx *c, const double *xprev, double t, double *b);

void or_rhs(const or_ctx *c, const double *xprev, double t, double *b) {
  if (c->geo == 1) {
    rhs_channel(c, xprev, t, b);
    return;
  }
  const int n = c->n, lat = c->bc != 0;
  const double h = c->h, mu = c->mu, cm = h * h / c->dt;
  /* u rows */
  for (int j = 0; j < n; ++j) {
    double y = 1.0 + (j + 0.5) * h;
    for (int i = 0; i <= n; ++i) {
      int64_t k = ix_u(n, i, j);
      double x = i * h;
      if ((i == 0 || i == n) && !lat) { b[k] = dat_u(c, x, y, t); continue; }
      if (i == 0 || i == n) {                   /* traction side, half control volume */
        const int rt = i == n;
        const double sg = rt ? -1.0 : 1.0;
        double s = 0.5 * cm * xprev[k] + 0.5 * h * h * dat_fx(c, x, y, t) + sg * h * side_p(c, rt, y, t);
        if (j < n - 1) s -= sg * mu * side_v(c, rt, 1.0 + (j + 1) * h, t);
        else s += mu * dat_u(c, x, 2.0, t) + sg * mu * (dat_v(c, x + sg * 0.5 * h, 2.0, t) - dat_v(c, x, 2.0, t));
        if (j > 0) s += sg * mu * side_v(c, rt, 1.0 + j * h, t);
        else s += sg * h * bjs_w_side(c, i) * side_v(c, rt, 1.0, t);
        b[k] = s;
        continue;
      }
      double s = cm * xprev[k] + h * h * dat_fx(c, x, y, t);
      if (i == 1 && !lat) s += 2.0 * mu * dat_u(c, 0.0, y, t);
      if (i == n - 1 && !lat) s += 2.0 * mu * dat_u(c, 1.0, y, t);
      if (j == n - 1)
        s += 2.0 * mu * dat_u(c, x, 2.0, t) + mu * (dat_v(c, x + 0.5 * h, 2.0, t) - dat_v(c, x - 0.5 * h, 2.0, t));
      b[k] = s;
    }
  }
  /* v rows */
  for (int j = 0; j <= n; ++j) {
    double y = 1.0 + j * h;
    for (int i = 0; i < n; ++i) {
      int64_t k = ix_v(n, i, j);
      double x = (i + 0.5) * h;
      if (j == n) { b[k] = dat_v(c, x, 2.0, t); continue; }
      if (j == 0) {
        double s = 0.5 * cm * xprev[k] + 0.5 * h * h * dat_fy(c, x, 1.0, t);
        if (i == 0) {
          if (lat) s += h * bjs_w_side(c, 0) * side_v(c, 0, 1.0, t);
          else s += -mu * (dat_u(c, 0.0, 1.0 + 0.5 * h, t) - dat_u(c, 0.0, 1.0, t)) + mu * dat_v(c, 0.0, 1.0, t);
        }
        if (i == n - 1) {
          if (lat) s += h * bjs_w_side(c, n) * side_v(c, 1, 1.0, t);
          else s += mu * (dat_u(c, 1.0, 1.0 + 0.5 * h, t) - dat_u(c, 1.0, 1.0, t)) + mu * dat_v(c, 1.0, 1.0, t);
        }
        b[k] = s;
        continue;
      }
      double s = cm * xprev[k] + h * h * dat_fy(c, x, y, t);
      if (j == n - 1) s += 2.0 * mu * dat_v(c, x, 2.0, t);
      if (i == 0) {
        if (lat) s += 2.0 * mu * side_v(c, 0, y, t);
        else s += 2.0 * mu * dat_v(c, 0.0, y, t) - mu * (dat_u(c, 0.0, y + 0.5 * h, t) - dat_u(c, 0.0, y - 0.5 * h, t));
      }
      if (i == n - 1) {
        if (lat) s += 2.0 * mu * side_v(c, 1, y, t);
        else s += 2.0 * mu * dat_v(c, 1.0, y, t) + mu * (dat_u(c, 1.0, y + 0.5 * h, t) - dat_u(c, 1.0, y - 0.5 * h, t));
      }
      b[k] = s;
    }
  }
  /* continuity rows */
  for (int j = 0; j < n; ++j) {
    double y = 1.0 + (j + 0.5) * h;
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      if (i == 0 && !lat) s += h * dat_u(c, 0.0, y, t);
      if (i == n - 1 && !lat) s -= h * dat_u(c, 1.0, y, t);
      if (j == n - 1) s -= h * dat_v(c, (i + 0.5) * h, 2.0, t);
      b[ix_pf(n, i, j)] = s;
    }
  }
  /* Darcy rows: no source; Dirichlet pressure at y = 0 */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      if (j == 0) s += 2.0 * kc(c, i, 0) / c->mu * dat_ppm(c, (i + 0.5) * h, 0.0, t);
      b[ix_pm(n, i, j)] = s;
    }
}


/* Right-hand side of the channel geometry (geo 1): the square's terms with
   the data of the walls beside Gamma (velocity on the floor faces and at the
   floor corners) moved in as the elimination of their identity rows asks.
   Ends: x = -1 (left), x = 2 (right). */
static double ch_side_p(const or_ctx *c, int right, double y, double t) {
  if (c->bc == 2) return right ? 0.0 : or_p_in(c->dp, c->tend, t);
  const double x = right ? 2.0 : -1.0;
  const double ux = OR_PI * cos(OR_PI * x) * mms_dphi(y) * (1.0 + t);
  return or_mms_pff(x, y, t, c->mu) - 2.0 * c->mu * ux;
}
static double ch_side_v(const or_ctx *c, int right, double y, double t) {
  return c->bc == 2 ? 0.0 : or_mms_v(right ? 2.0 : -1.0, y, t);
}

static void rhs_channel(const or_ctx *c, const double *xprev, double t, double *b) {
  const int n = c->n, NX = c->nx, lat = c->bc != 0;
  const double h = c->h, mu = c->mu, cm = h * h / c->dt;
  const double xl = -1.0, xr = 2.0;
  /* u rows */
  for (int j = 0; j < n; ++j) {
    const double y = 1.0 + (j + 0.5) * h;
    for (int i = 0; i <= NX; ++i) {
      const int64_t k = chu(c, i, j);
      const double x = chx(c, i);
      if ((i == 0 || i == NX) && !lat) { b[k] = dat_u(c, x, y, t); continue; }
      if (i == 0 || i == NX) {                   /* traction end */
        const int rt = i == NX;
        const double sg = rt ? -1.0 : 1.0;
        double s = 0.5 * cm * xprev[k] + 0.5 * h * h * dat_fx(c, x, y, t) + sg * h * ch_side_p(c, rt, y, t);
        if (j < n - 1) s -= sg * mu * ch_side_v(c, rt, 1.0 + (j + 1) * h, t);
        else s += mu * dat_u(c, x, 2.0, t) + sg * mu * (dat_v(c, x + sg * 0.5 * h, 2.0, t) - dat_v(c, x, 2.0, t));
        if (j > 0) s += sg * mu * ch_side_v(c, rt, 1.0 + j * h, t);
        else s += mu * dat_u(c, x, 1.0, t) - sg * mu * (dat_v(c, x + sg * 0.5 * h, 1.0, t) - dat_v(c, x, 1.0, t));
        b[k] = s;
        continue;
      }
      double s = cm * xprev[k] + h * h * dat_fx(c, x, y, t);
      if (i == 1 && !lat) s += 2.0 * mu * dat_u(c, xl, y, t);
      if (i == NX - 1 && !lat) s += 2.0 * mu * dat_u(c, xr, y, t);
      if (j == n - 1)
        s += 2.0 * mu * dat_u(c, x, 2.0, t) + mu * (dat_v(c, x + 0.5 * h, 2.0, t) - dat_v(c, x - 0.5 * h, 2.0, t));
      if (j == 0) {
        if (i >= c->iw && i <= c->iw + n) {       /* BJS corner: a wall face beside the slip is data */
          const double w = bjs_w_ch(c, i);
          if (!on_gamma(c, i)) s -= w * h * dat_v(c, x + 0.5 * h, 1.0, t);
          if (!on_gamma(c, i - 1)) s += w * h * dat_v(c, x - 0.5 * h, 1.0, t);
        } else {                                  /* floor wall at half distance */
          s += 2.0 * mu * dat_u(c, x, 1.0, t) - mu * (dat_v(c, x + 0.5 * h, 1.0, t) - dat_v(c, x - 0.5 * h, 1.0, t));
        }
      }
      b[k] = s;
    }
  }
  /* v rows */
  for (int j = 0; j <= n; ++j) {
    const double y = 1.0 + j * h;
    for (int i = 0; i < NX; ++i) {
      const int64_t k = chv(c, i, j);
      const double x = chx(c, i) + 0.5 * h;
      if (j == n) { b[k] = dat_v(c, x, 2.0, t); continue; }
      if (j == 0 && !on_gamma(c, i)) { b[k] = dat_v(c, x, 1.0, t); continue; }
      if (j == 0) {
        double s = 0.5 * cm * xprev[k] + 0.5 * h * h * dat_fy(c, x, 1.0, t);
        if (!on_gamma(c, i - 1)) s += 0.5 * h * bjs_w_ch(c, i) * dat_v(c, x - h, 1.0, t);
        if (!on_gamma(c, i + 1)) s += 0.5 * h * bjs_w_ch(c, i + 1) * dat_v(c, x + h, 1.0, t);
        b[k] = s;
        continue;
      }
      double s = cm * xprev[k] + h * h * dat_fy(c, x, y, t);
      if (j == n - 1) s += 2.0 * mu * dat_v(c, x, 2.0, t);
      if (j == 1 && !on_gamma(c, i)) s += 2.0 * mu * dat_v(c, x, 1.0, t);
      if (i == 0) {
        if (lat) s += 2.0 * mu * ch_side_v(c, 0, y, t);
        else s += 2.0 * mu * dat_v(c, xl, y, t) - mu * (dat_u(c, xl, y + 0.5 * h, t) - dat_u(c, xl, y - 0.5 * h, t));
      }
      if (i == NX - 1) {
        if (lat) s += 2.0 * mu * ch_side_v(c, 1, y, t);
        else s += 2.0 * mu * dat_v(c, xr, y, t) + mu * (dat_u(c, xr, y + 0.5 * h, t) - dat_u(c, xr, y - 0.5 * h, t));
      }
      b[k] = s;
    }
  }
  /* continuity rows */
  for (int j = 0; j < n; ++j) {
    const double y = 1.0 + (j + 0.5) * h;
    for (int i = 0; i < NX; ++i) {
      double s = 0.0;
      const double x = chx(c, i) + 0.5 * h;
      if (i == 0 && !lat) s += h * dat_u(c, xl, y, t);
      if (i == NX - 1 && !lat) s -= h * dat_u(c, xr, y, t);
      if (j == n - 1) s -= h * dat_v(c, x, 2.0, t);
      if (j == 0 && !on_gamma(c, i)) s += h * dat_v(c, x, 1.0, t);
      b[chp(c, i, j)] = s;
    }
  }
  /* Darcy rows */
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) {
      double s = 0.0;
      if (j == 0) s += 2.0 * kc(c, i, 0) / c->mu * dat_ppm(c, (i + 0.5) * h, 0.0, t);
      b[chm(c, i, j)] = s;
    }
}

/* The manufactured solution on the channel's unknowns (geo 1) or the square's (geo 0). */
void or_exact_geo(int n, double t, double mu, int geo, double *x) {
  if (geo != 1) {
    or_exact(n, t, mu, x);
    return;
  }
  or_ctx g;
  memset(&g, 0, sizeof(g));
  g.n = n; g.nx = 3 * n; g.iw = n; g.h = 1.0 / n; g.geo = 1;
  const double h = g.h;
  for (int j = 0; j < n; ++j)
    for (int i = 0; i <= g.nx; ++i) x[chu(&g, i, j)] = or_mms_u(chx(&g, i), 1.0 + (j + 0.5) * h, t);
  for (int j = 0; j <= n; ++j)
    for (int i = 0; i < g.nx; ++i) x[chv(&g, i, j)] = or_mms_v(chx(&g, i) + 0.5 * h, 1.0 + j * h, t);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < g.nx; ++i) x[chp(&g, i, j)] = or_mms_pff(chx(&g, i) + 0.5 * h, 1.0 + (j + 0.5) * h, t, mu);
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) x[chm(&g, i, j)] = or_mms_ppm((i + 0.5) * h, (j + 0.5) * h, t);
}

/* ------------------------------------------------------------------------ */
/* Banded LU with partial pivoting                                           */
/* Unknowns are re-ordered by height (then by x) so that A is banded with    */
/* bandwidth about 3n; the same permutation is applied to rows and columns.  */
/* ------------------------------------------------------------------------ */
static int64_t sort_key_channel(const or_ctx *c, int64_t k) {
  /* the square's ordering over the channel: pm cells at the x of the free-flow columns above them */
  const int n = c->n, NX = c->nx;
  const int64_t nu = (int64_t)n * (NX + 1), nv = (int64_t)NX * (n + 1), np = (int64_t)NX * n;
  const int64_t W = 2 * (int64_t)NX + 2;
  int64_t lev, xp, kind;
  if (k < nu) { int64_t j = k / (NX + 1), i = k % (NX + 1); lev = 2 * n + 2 * j + 1; xp = 2 * i; kind = 0; }
  else if (k < nu + nv) { k -= nu; int64_t j = k / NX, i = k % NX; lev = 2 * n + 2 * j; xp = 2 * i + 1; kind = 1; }
  else if (k < nu + nv + np) { k -= nu + nv; int64_t j = k / NX, i = k % NX; lev = 2 * n + 2 * j + 1; xp = 2 * i + 1; kind = 2; }
  else { k -= nu + nv + np; int64_t j = k / n, i = k % n; lev = 2 * j + 1; xp = 2 * (i + c->iw) + 1; kind = 3; }
  return (lev * W + xp) * 4 + kind;
}

static int64_t sort_key(int n, int64_t k) {
  /* key = (level in units of h/2 from y = 0) * (2n+2) + (x in units of h/2) */
  int64_t nu = (int64_t)n * (n + 1), np = (int64_t)n * n;
  int64_t W = 2 * (int64_t)n + 2, lev, xp, kind;
  if (k < nu) { int64_t j = k / (n + 1), i = k % (n + 1); lev = 2 * n + 2 * j + 1; xp = 2 * i; kind = 0; }
  else if (k < 2 * nu) { k -= nu; int64_t j = k / n, i = k % n; lev = 2 * n + 2 * j; xp = 2 * i + 1; kind = 1; }
  else if (k < 2 * nu + np) { k -= 2 * nu; int64_t j = k / n, i = k % n; lev = 2 * n + 2 * j + 1; xp = 2 * i + 1; kind = 2; }
  else { k -= 2 * nu + np; int64_t j = k / n, i = k % n; lev = 2 * j + 1; xp = 2 * i + 1; kind = 3; }
  return (lev * W + xp) * 4 + kind;
}

static int64_t *g_keys;
static int cmp_keys(const void *a, const void *b) {
  int64_t ka = g_keys[*(const int32_t *)a], kb = g_keys[*(const int32_t *)b];
  return (ka > kb) - (ka < kb);
}

int or_factor(or_ctx *c) {
  const int64_t N = c->ndof;
  free(c->perm); free(c->iperm); free(c->ab); free(c->ipiv);
  c->perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  c->iperm = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  int64_t *keys = (int64_t *)malloc(sizeof(int64_t) * (size_t)N);
  for (int64_t k = 0; k < N; ++k) {
    keys[k] = c->geo == 1 ? sort_key_channel(c, k) : sort_key(c->n, k);
    c->perm[k] = (int32_t)k;
  }
  g_keys = keys;
  qsort(c->perm, (size_t)N, sizeof(int32_t), cmp_keys);
  g_keys = NULL;
  free(keys);
  for (int64_t k = 0; k < N; ++k) c->iperm[c->perm[k]] = (int32_t)k;
  int kl = 0, ku = 0;
  for (int64_t r = 0; r < N; ++r)
    for (int64_t k = c->rowptr[r]; k < c->rowptr[r + 1]; ++k) {
      int64_t d = (int64_t)c->iperm[r] - c->iperm[c->col[k]];
      if (d > kl) kl = (int)d;
      if (-d > ku) ku = (int)(-d);
    }
  c->kl = kl; c->ku = ku;
  c->ldab = 2 * (int64_t)kl + ku + 1;
  const int64_t ld = c->ldab, kv = kl + ku; /* row of the diagonal inside a band column */
  c->ab = (double *)calloc((size_t)(ld * N), sizeof(double));
  c->ipiv = (int32_t *)malloc(sizeof(int32_t) * (size_t)N);
  if (!c->ab || !c->ipiv) return -1;
  double *ab = c->ab;
#define AB(i, j) ab[(kv + (i) - (j)) + (int64_t)(j) * ld]
  for (int64_t r = 0; r < N; ++r)
    for (int64_t k = c->rowptr[r]; k < c->rowptr[r + 1]; ++k) AB(c->iperm[r], c->iperm[c->col[k]]) += c->val[k];
  int64_t ju = 0;
  int info = 0;
  for (int64_t j = 0; j < N; ++j) {
    int64_t km = kl < N - 1 - j ? kl : N - 1 - j;
    int64_t p = 0; double amax = fabs(AB(j, j));
    for (int64_t i = 1; i <= km; ++i) { double a = fabs(AB(j + i, j)); if (a > amax) { amax = a; p = i; } }
    c->ipiv[j] = (int32_t)(j + p);
    if (amax == 0.0) { if (!info) info = (int)(j + 1); continue; }
    int64_t jend = j + ku + p; if (jend > N - 1) jend = N - 1;
    if (jend > ju) ju = jend;
    if (p != 0)
      for (int64_t jj = j; jj <= ju; ++jj) { double t = AB(j, jj); AB(j, jj) = AB(j + p, jj); AB(j + p, jj) = t; }
    double rpiv = 1.0 / AB(j, j);
    for (int64_t i = 1; i <= km; ++i) AB(j + i, j) *= rpiv;
    for (int64_t jj = j + 1; jj <= ju; ++jj) {
      double a = AB(j, jj);
      if (a == 0.0) continue;
      double *colp = &AB(j + 1, jj);
      const double *lp = &AB(j + 1, j);
      for (int64_t i = 0; i < km; ++i) colp[i] -= lp[i] * a;
    }
  }
#undef AB
  c->factored = (info == 0);
  return info;
}

/* Solve A x = b with the factors of or_factor. */
int or_solve(const or_ctx *c, const double *b, double *x) {
  if (!c->factored) return -1;
  const int64_t N = c->ndof, ld = c->ldab, kl = c->kl, kv = c->kl + c->ku;
  const double *ab = c->ab;
#define AB(i, j) ab[(kv + (i) - (j)) + (int64_t)(j) * ld]
  double *y = (double *)malloc(sizeof(double) * (size_t)N);
  for (int64_t k = 0; k < N; ++k) y[k] = b[c->perm[k]];
  for (int64_t j = 0; j < N; ++j) { /* L y = P b */
    int64_t p = c->ipiv[j];
    if (p != j) { double t = y[j]; y[j] = y[p]; y[p] = t; }
    int64_t km = kl < N - 1 - j ? kl : N - 1 - j;
    double yj = y[j];
    for (int64_t i = 1; i <= km; ++i) y[j + i] -= AB(j + i, j) * yj;
  }
  for (int64_t j = N - 1; j >= 0; --j) { /* U x = y, U has bandwidth kl + ku */
    y[j] /= AB(j, j);
    int64_t i0 = j - kv < 0 ? 0 : j - kv;
    double yj = y[j];
    for (int64_t i = i0; i < j; ++i) y[i] -= AB(i, j) * yj;
  }
#undef AB
  for (int64_t k = 0; k < N; ++k) x[c->perm[k]] = y[k];
  free(y);
  return 0;
}

int or_bandwidth(const or_ctx *c, int *kl, int *ku) { *kl = c->kl; *ku = c->ku; return c->factored; }

/* r = b - A x, returns ||r||_2 */
double or_residual(const or_ctx *c, const double *x, const double *b, double *r) {
  double s = 0.0;
  for (int64_t row = 0; row < c->ndof; ++row) {
    double a = b[row];
    for (int64_t k = c->rowptr[row]; k < c->rowptr[row + 1]; ++k) a -= c->val[k] * x[c->col[k]];
    if (r) r[row] = a;
    s += a * a;
  }
  return sqrt(s);
}

/* Run nsteps implicit-Euler steps from state x (in place) starting at time t0.
   The factorisation must exist.  Returns 0 on success. */
int or_run(const or_ctx *c, double *x, double t0, int nsteps) {
  double *b = (double *)malloc(sizeof(double) * (size_t)c->ndof);
  int rc = 0;
  for (int s = 0; s < nsteps && rc == 0; ++s) {
    double t = t0 + (s + 1) * c->dt;
    or_rhs(c, x, t, b);
    rc = or_solve(c, b, x);
  }
  free(b);
  return rc;
}
