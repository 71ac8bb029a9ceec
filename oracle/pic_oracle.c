/*
 * FP64 CPU oracle of the boosted-frame electromagnetic PIC step, 2-1/2D (x,z).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library. The product
 * path (the CUDA library behind include/pic.h) neither links nor calls it, and
 * this file includes no header of the product.
 *
 * It restates, in plain loops and in the paper's order, the method of
 * J.-L. Vay, C.G.R. Geddes, E. Cormier-Michel, D.P. Grote, "Modeling laser
 * wakefield accelerators in a Lorentz boosted frame" (arXiv:1009.2727):
 *   - Sec. 4.2  tunable (Cole-Karkkainen) Faraday update, Eq. Faraday/Ampere,
 *               2D reduction of the enlarged operator;
 *   - Sec. 4.3  Friedman damping, Eq. Faraday_Friedman;
 *   - Sec. 4.1  multi-pass bilinear filter with compensation, Eq. 3ptfilter
 *               and its strided form;
 *   - App. II   split-field PML with the enlarged stencil, Eq. PML_stencil;
 *   - Sec. 4.2.2 Esirkepov charge-conserving deposition (ref. Esirkepov 2001);
 *   - Sec. 5    cubic-spline shapes, energy-conserving gather from the Yee
 *               locations;
 *   - Sec. 3.1  particle and laser input through planes (boosted frame);
 *   - Sec. 3.2  lab-frame "stations"/snapshots by interpolation.
 * The relativistic Boris push is the textbook scheme (Birdsall & Langdon,
 * cited by the paper). Wherever the paper is silent or garbled, the reading
 * used here is the one listed in the project's design notes (PR-n numbers in
 * comments refer to those readings).
 *
 * Every array is double precision. Nothing here is blocked, fused or
 * reordered beyond what the method states. Compile with -ffp-contract=off so
 * that results do not depend on the host's FMA contraction.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 */
#define O_C 299792458.0
#define O_QE 1.602176634e-19
#define O_ME 9.1093837015e-31
#define O_EPS0 8.8541878128e-12
#define O_MU0 (1.0 / (O_EPS0 * O_C * O_C))
#define O_PI 3.14159265358979323846

/* component ids: E, B, J */
enum { OEX = 0, OEY, OEZ, OBX, OBY, OBZ, OJX, OJY, OJZ, ONCOMP };

/* ------------------------------------------------------------------ */
/* configuration (this file's own definition; not shared with the GPU) */
typedef struct {
  int nx, nz;                 /* cells */
  double dz_lab;              /* lab longitudinal cell [m]; boosted dz = (1+beta) gamma dz_lab (Sec. 5.1.1) */
  double dx;                  /* transverse cell [m] (frame invariant) */
  double gamma_boost;         /* >= 1 */
  double courant;             /* dt = courant * dt_CFL when dt_override <= 0 */
  double dt_override;
  double ck_alpha, ck_beta, ck_gamma; /* 3D coefficients of Table CKcoefs */
  double theta;               /* Friedman damping, 0 <= theta <= 1 */
  int pml_cells;
  double pml_sigma_max;       /* sigma_m in units of c/delta (paper: 4) */
  double pml_delta;           /* Delta in cells (paper: 5) */
  double pml_power;           /* n (paper: 2) */
  int pml_xi_exp;             /* 1: xi = exp(-sigma dt); 0: (1 - sigma dt/2)/(1 + sigma dt/2) */
  int filter_passes, filter_stride, filter_compensate, filter_J, filter_gather;
  int order;                  /* shape order 1 or 3 */
  int particle_guard;         /* cells between PML and particle domain; <0 => default */
  int periodic_x, periodic_z; /* fields only (test option) */
  int moving_window;
  double window_beta;
  int filter_strides[4];      /* > 0: the wide-band filter of Sec. 4.1, the product over these strides of
                                 (n passes + compensation) at each stride, e.g. 1,2,3 for S(1:2:3); else 0 */
  int gather_nodal;           /* 0: 'energy conserving' gather from the Yee locations (Sec. 5);
                                 1: 'momentum conserving': the fields are first interpolated to the nodes */
  int beam_self;              /* 1: the test beam's frozen and active particles deposit their current
                                 (Sec. 3.1.1: the charge and current of the frozen particles keep the fields
                                 at the injection plane consistent); 0: test particles */
} orc_config;

typedef struct {
  double n0;                  /* lab electron density [m^-3] */
  double z_start_lab;         /* lab position where the ramp starts [m] */
  double ramp_lab;            /* linear ramp length (lab) [m] */
  double length_lab;          /* plateau length (lab) [m]; <= 0 means unbounded */
  int ppc_x, ppc_z;
  int ions;                   /* 1: ions fixed in the lab (ballistic in the boosted frame) */
} orc_plasma;

typedef struct {
  double lambda0, a0, w0, tau_fwhm, t_peak, x_center, phase;
  double z_antenna;           /* computational-frame position at t'=0 [m] */
  double beta_s;              /* antenna-plane velocity / c in the computational frame */
} orc_laser;

typedef struct {
  double *x, *z, *ux, *uy, *uz, *w;
  uint32_t *id;
  int *alive;
  /* beam-only */
  double *tc, *zf0, *uxb, *uyb, *uzb; int *active;
  /* ions: lattice position (m + 1/2) h of the row, fixed in the lab */
  double *zl;
  long n, cap;
  double q, m;
} orc_species;

typedef struct {
  orc_config c;
  double dx, dz, dt, gamma, beta;
  double a2, b2;              /* 2D reduced CK coefficients (PR-3) */
  int nxp, nzp;               /* nx+1, nz+1 */
  long ncell;
  double *F[ONCOMP];
  double *Ep[3], *Eb[3], *Ee[3];  /* Friedman E^{n-1}, E-bar, E_eff */
  double *Bold[3];
  double *fE[3], *fB[3];          /* filtered copies for the gather */
  double *Byx, *Byz, *Eyx, *Eyz;  /* split PML parts */
  double *tmp;
  double *sx_int, *sx_half, *sz_int, *sz_half; /* sigma at integer / half positions */
  double z0;                  /* grid origin (moving window) */
  long shifts;
  long step;
  int gx_lo, gx_hi, gz_lo, gz_hi; /* particle domain in cells */
  orc_species sp[3];          /* 0 electrons, 1 ions, 2 test beam */
  orc_plasma pl; int has_plasma;
  long row_next_e, nxl;       /* next lattice row to inject; x-lattice size */
  double h_row;
  orc_laser las; int has_laser;
  double beam_vbar; int has_beam;
  /* lab-frame sample rows (back-transformed diagnostics) */
  int nrows; double *rzL, *rtL, *rout; int *rdone;
  /* external current source (test hook for the App. I source problems) */
  double *ext[3]; int ext_alternate; double *ext_prof; long ext_nprof;
} orc_sim;

/* ------------------------------------------------------------------ */
/* B-spline shape of order 1 and 3, by definition (Sec. 4: cubic splines). */
double orc_shape(int order, double s) {
  double a = fabs(s);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { double t = 2.0 - a; return t * t * t / 6.0; }
  return 0.0;
}

/* ------------------------------------------------------------------ */
/* Stability limit of the tunable solver (Eq. cfl) and its 2D restriction
 * (PR-3), times the Friedman factor sqrt((2+theta)/(2+3theta)) (Sec. 4.3). */
double orc_cfl_3d(double a, double b, double g, double dx, double dy, double dz, double theta) {
  double kx = 1.0 / (dx * dx), ky = 1.0 / (dy * dy), kz = 1.0 / (dz * dz);
  double m = dx < dy ? dx : dy; if (dz < m) m = dz;
  double pair = kx + ky; if (kx + kz > pair) pair = kx + kz; if (ky + kz > pair) pair = ky + kz;
  double t1 = (a - 4.0 * g) * pair, t2 = (a - 4.0 * b + 4.0 * g) * (kx + ky + kz);
  double r = m;
  if (t1 > 0 && 1.0 / sqrt(t1) < r) r = 1.0 / sqrt(t1);
  if (t2 > 0 && 1.0 / sqrt(t2) < r) r = 1.0 / sqrt(t2);
  return r / O_C * sqrt((2.0 + theta) / (2.0 + 3.0 * theta));
}

double orc_cfl_2d(double a, double b, double g, double dx, double dz, double theta) {
  (void)b; /* the 2D limit involves alpha2 - 2 beta2 = alpha - 4 gamma only */
  double kx = 1.0 / (dx * dx), kz = 1.0 / (dz * dz);
  double mx = kx > kz ? kx : kz;
  double t = (a - 4.0 * g) * (kx + kz);
  if (t > mx) mx = t;
  return 1.0 / sqrt(mx) / O_C * sqrt((2.0 + theta) / (2.0 + 3.0 * theta));
}

/* ------------------------------------------------------------------ */
/* One pass of the 3-point filter with stride s (Eq. 3ptfilter_stride) on a
 * 1D line, zero outside [0,n) unless periodic. out may not alias in. */
void orc_filter_line(const double* in, double* out, int n, int s, double alpha, int periodic) {
  for (int j = 0; j < n; j++) {
    double l = 0.0, r = 0.0;
    int jl = j - s, jr = j + s;
    if (periodic) { jl = ((jl % n) + n) % n; jr = jr % n; l = in[jl]; r = in[jr]; }
    else { if (jl >= 0) l = in[jl]; if (jr < n) r = in[jr]; }
    out[j] = alpha * in[j] + (1.0 - alpha) * 0.5 * (l + r);
  }
}

/* ------------------------------------------------------------------ */
/* Relativistic Boris push (textbook, Birdsall & Langdon): u = gamma v.
 * u^{n-1/2} -> u^{n+1/2} with fields at integer time. */
void orc_boris(double* u, const double* E, const double* B, double q, double m, double dt) {
  double k = q * dt / (2.0 * m);
  double um[3] = { u[0] + k * E[0], u[1] + k * E[1], u[2] + k * E[2] };
  double g = sqrt(1.0 + (um[0] * um[0] + um[1] * um[1] + um[2] * um[2]) / (O_C * O_C));
  double t[3] = { k * B[0] / g, k * B[1] / g, k * B[2] / g };
  double t2 = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
  double s[3] = { 2.0 * t[0] / (1.0 + t2), 2.0 * t[1] / (1.0 + t2), 2.0 * t[2] / (1.0 + t2) };
  double up[3] = { um[0] + (um[1] * t[2] - um[2] * t[1]),
                   um[1] + (um[2] * t[0] - um[0] * t[2]),
                   um[2] + (um[0] * t[1] - um[1] * t[0]) };
  double pl[3] = { um[0] + (up[1] * s[2] - up[2] * s[1]),
                   um[1] + (up[2] * s[0] - up[0] * s[2]),
                   um[2] + (up[0] * s[1] - up[1] * s[0]) };
  u[0] = pl[0] + k * E[0]; u[1] = pl[1] + k * E[1]; u[2] = pl[2] + k * E[2];
}

/* ------------------------------------------------------------------ */
/* grid access helpers */
static inline long IDX(const orc_sim* s, int i, int k) { return (long)i * s->nzp + k; }

static double rd(const orc_sim* s, const double* F, int i, int k) {
  if (s->c.periodic_x) { i %= s->c.nx; if (i < 0) i += s->c.nx; }
  if (s->c.periodic_z) { k %= s->c.nz; if (k < 0) k += s->c.nz; }
  if (i < 0 || i > s->c.nx || k < 0 || k > s->c.nz) return 0.0;
  return F[IDX(s, i, k)];
}

/* stagger (in cells) of each component: E/J and B on the Yee mesh (PML stencil index pattern, App. II) */
static const double STX[ONCOMP] = { 0.5, 0.0, 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0 };
static const double STZ[ONCOMP] = { 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 0.5 };

/* valid index range of a component (PEC walls: tangential E vanishes on the boundary) */
static void vrange(const orc_sim* s, int comp, int* i0, int* i1, int* k0, int* k1) {
  int c = comp >= OJX ? comp - OJX : comp;
  int nx = s->c.nx, nz = s->c.nz;
  switch (c) {
    case OEX: *i0 = 0; *i1 = nx - 1; *k0 = 1; *k1 = nz - 1; break;
    case OEY: *i0 = 1; *i1 = nx - 1; *k0 = 1; *k1 = nz - 1; break;
    case OEZ: *i0 = 1; *i1 = nx - 1; *k0 = 0; *k1 = nz - 1; break;
    case OBX: *i0 = 0; *i1 = nx;     *k0 = 0; *k1 = nz - 1; break;
    case OBY: *i0 = 0; *i1 = nx - 1; *k0 = 0; *k1 = nz - 1; break;
    default:  *i0 = 0; *i1 = nx - 1; *k0 = 0; *k1 = nz;     break;
  }
  if (s->c.periodic_x) { *i0 = 0; *i1 = nx - 1; }
  if (s->c.periodic_z) { *k0 = 0; *k1 = nz - 1; }
}

/* PML absorption profile, App. II: sigma = sigma_m (d/Delta)^n, d = depth in
 * cells at the component's own (staggered) position (PR-18). */
static double pml_sigma(const orc_sim* s, double pos, int n, double d_cell) {
  int L = s->c.pml_cells;
  if (L <= 0) return 0.0;
  double d = 0.0;
  if (pos < L) d = L - pos;
  if (pos > n - L) d = pos - (n - L);
  if (d <= 0.0) return 0.0;
  return s->c.pml_sigma_max * O_C / d_cell * pow(d / s->c.pml_delta, s->c.pml_power);
}

static double pml_xi(const orc_sim* s, double sig) {
  if (s->c.pml_xi_exp) return exp(-sig * s->dt);
  return (1.0 - 0.5 * sig * s->dt) / (1.0 + 0.5 * sig * s->dt);
}

/* (1 - xi)/sigma, which tends to dt as sigma -> 0 */
static double pml_coef(const orc_sim* s, double sig) {
  if (sig <= 0.0) return s->dt;
  return (1.0 - pml_xi(s, sig)) / sig;
}

/* ------------------------------------------------------------------ */
/* Enlarged difference operators of Sec. 4.2 restricted to d/dy = 0 (PR-2,
 * PR-3): Delta*_z = (a2 + b2 S_x) Delta_z with S_x the sum of the two
 * x-neighbours at one full cell (the offsets fixed by Eq. num_disp), a2 =
 * alpha + 2 beta, b2 = beta + 2 gamma. Result sits half a cell above k. */
static double dstar_z(const orc_sim* s, const double* F, int i, int k) {
  double c0 = rd(s, F, i, k + 1) - rd(s, F, i, k);
  double cp = rd(s, F, i + 1, k + 1) - rd(s, F, i + 1, k);
  double cm = rd(s, F, i - 1, k + 1) - rd(s, F, i - 1, k);
  return (s->a2 * c0 + s->b2 * (cp + cm)) / s->dz;
}

static double dstar_x(const orc_sim* s, const double* F, int i, int k) {
  double c0 = rd(s, F, i + 1, k) - rd(s, F, i, k);
  double cp = rd(s, F, i + 1, k + 1) - rd(s, F, i, k + 1);
  double cm = rd(s, F, i + 1, k - 1) - rd(s, F, i, k - 1);
  return (s->a2 * c0 + s->b2 * (cp + cm)) / s->dx;
}

/* ------------------------------------------------------------------ */
/* Faraday with the enlarged stencil (Eq. Faraday), Friedman time filter on E
 * (Eq. Faraday_Friedman, PR-1 indexing) and the split-field PML for B
 * (Eq. PML_stencil). Advances B^{n-1/2} -> B^{n+1/2} using E^n. */
static void faraday(orc_sim* s) {
  double th = s->c.theta;
  long N = s->ncell;
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < N; p++)
      s->Ee[c][p] = (1.0 + th / 4.0) * s->F[OEX + c][p] - 0.5 * s->Ep[c][p] + (0.5 - th / 4.0) * s->Eb[c][p];
  for (int c = 0; c < 3; c++) memcpy(s->Bold[c], s->F[OBX + c], sizeof(double) * N);
  const double *Ex = s->Ee[0], *Ey = s->Ee[1], *Ez = s->Ee[2];
  double *Bx = s->F[OBX], *By = s->F[OBY], *Bz = s->F[OBZ];
  int i0, i1, k0, k1;
  /* Bx at (i, k+1/2): dBx/dt = d(Ey)/dz */
  vrange(s, OBX, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double d = dstar_z(s, Ey, i, k);
      double sz = s->sz_half[k];
      long p = IDX(s, i, k);
      if (sz > 0.0) Bx[p] = pml_xi(s, sz) * Bx[p] + pml_coef(s, sz) * d;
      else Bx[p] = Bx[p] + s->dt * d;
    }
  /* Bz at (i+1/2, k): dBz/dt = -d(Ey)/dx */
  vrange(s, OBZ, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double d = dstar_x(s, Ey, i, k);
      double sx = s->sx_half[i];
      long p = IDX(s, i, k);
      if (sx > 0.0) Bz[p] = pml_xi(s, sx) * Bz[p] - pml_coef(s, sx) * d;
      else Bz[p] = Bz[p] - s->dt * d;
    }
  /* By at (i+1/2, k+1/2): dBy/dt = -d(Ex)/dz + d(Ez)/dx, split By = Byx + Byz in the PML */
  vrange(s, OBY, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double a = dstar_z(s, Ex, i, k);
      double b = dstar_x(s, Ez, i, k);
      double sx = s->sx_half[i], sz = s->sz_half[k];
      long p = IDX(s, i, k);
      if (sx > 0.0 || sz > 0.0) {
        s->Byz[p] = pml_xi(s, sz) * s->Byz[p] - pml_coef(s, sz) * a;
        s->Byx[p] = pml_xi(s, sx) * s->Byx[p] + pml_coef(s, sx) * b;
        By[p] = s->Byx[p] + s->Byz[p];
      } else {
        By[p] = By[p] - s->dt * (a - b);
      }
    }
  /* Friedman history: E-bar <- (1 - theta/2) E^n + (theta/2) E-bar, E^{n-1} <- E^n */
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < N; p++) {
      s->Eb[c][p] = (1.0 - th / 2.0) * s->F[OEX + c][p] + (th / 2.0) * s->Eb[c][p];
      s->Ep[c][p] = s->F[OEX + c][p];
    }
}

/* Ampere with the standard (Yee) operator (Eq. Ampere) and the split-field PML
 * for E (Eq. PML_stencil). Advances E^n -> E^{n+1} with B^{n+1/2}, J^{n+1/2}.
 * No current is applied inside the PML, where the particle guard keeps J zero. */
static void ampere(orc_sim* s) {
  const double c2 = O_C * O_C, dt = s->dt;
  const double *Bx = s->F[OBX], *By = s->F[OBY], *Bz = s->F[OBZ];
  double *Ex = s->F[OEX], *Ey = s->F[OEY], *Ez = s->F[OEZ];
  const double *Jx = s->F[OJX], *Jy = s->F[OJY], *Jz = s->F[OJZ];
  int i0, i1, k0, k1;
  vrange(s, OEX, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double d = (rd(s, By, i, k) - rd(s, By, i, k - 1)) / s->dz;
      double sz = s->sz_int[k];
      long p = IDX(s, i, k);
      if (sz > 0.0) Ex[p] = pml_xi(s, sz) * Ex[p] - c2 * pml_coef(s, sz) * d;
      else Ex[p] = Ex[p] - dt * (c2 * d + Jx[p] / O_EPS0);
    }
  vrange(s, OEZ, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double d = (rd(s, By, i, k) - rd(s, By, i - 1, k)) / s->dx;
      double sx = s->sx_int[i];
      long p = IDX(s, i, k);
      if (sx > 0.0) Ez[p] = pml_xi(s, sx) * Ez[p] + c2 * pml_coef(s, sx) * d;
      else Ez[p] = Ez[p] + dt * (c2 * d - Jz[p] / O_EPS0);
    }
  vrange(s, OEY, &i0, &i1, &k0, &k1);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double dbx = (rd(s, Bx, i, k) - rd(s, Bx, i, k - 1)) / s->dz;
      double dbz = (rd(s, Bz, i, k) - rd(s, Bz, i - 1, k)) / s->dx;
      double sx = s->sx_int[i], sz = s->sz_int[k];
      long p = IDX(s, i, k);
      if (sx > 0.0 || sz > 0.0) {
        s->Eyz[p] = pml_xi(s, sz) * s->Eyz[p] + c2 * pml_coef(s, sz) * dbx;
        s->Eyx[p] = pml_xi(s, sx) * s->Eyx[p] - c2 * pml_coef(s, sx) * dbz;
        Ey[p] = s->Eyx[p] + s->Eyz[p];
      } else {
        Ey[p] = Ey[p] + dt * (c2 * (dbx - dbz) - Jy[p] / O_EPS0);
      }
    }
}

/* ------------------------------------------------------------------ */
/* Filter of Sec. 4.1 applied to one grid component: n bilinear passes
 * (alpha = 1/2) then, if requested, one compensation pass alpha_c = n/2 + 1,
 * all along x, then all along z (PR-5, PR-6). Zero outside the component's
 * valid range; the output is kept on the valid range after every pass. */
static void filter_pass_axis(orc_sim* s, int comp, double* F, int axis, int stride, double alpha) {
  int i0, i1, k0, k1;
  vrange(s, comp, &i0, &i1, &k0, &k1);
  double* out = s->tmp;
  memset(out, 0, sizeof(double) * s->ncell);
  for (int i = i0; i <= i1; i++)
    for (int k = k0; k <= k1; k++) {
      double l, r;
      if (axis == 0) { l = rd(s, F, i - stride, k); r = rd(s, F, i + stride, k); }
      else { l = rd(s, F, i, k - stride); r = rd(s, F, i, k + stride); }
      out[IDX(s, i, k)] = alpha * F[IDX(s, i, k)] + (1.0 - alpha) * 0.5 * (l + r);
    }
  memcpy(F, out, sizeof(double) * s->ncell);
}

/* With a stride set (Sec. 4.1, wide-band filters combining strides): along each axis, for each stride
 * of the set in turn, the n passes and the compensation pass at that stride. */
static void filter_component(orc_sim* s, int comp, double* F) {
  int n = s->c.filter_passes;
  int set[4] = { s->c.filter_stride, 0, 0, 0 };
  if (s->c.filter_strides[0] > 0) for (int q = 0; q < 4; q++) set[q] = s->c.filter_strides[q];
  for (int axis = 0; axis < 2; axis++)
    for (int q = 0; q < 4 && set[q] > 0; q++) {
      for (int p = 0; p < n; p++) filter_pass_axis(s, comp, F, axis, set[q], 0.5);
      if (s->c.filter_compensate) filter_pass_axis(s, comp, F, axis, set[q], 0.5 * n + 1.0);
    }
}

/* 'Momentum conserving' gather (Sec. 5, scan of the time step): the staggered gather copy of a component
 * is first interpolated to the grid nodes, as the mean of its two nearest values along each half-integer
 * axis (four for a component staggered along x and z); values off the grid count as zero. */
static void to_nodes(orc_sim* s, int comp, double* F) {
  int hx = STX[comp] != 0.0, hz = STZ[comp] != 0.0;
  double* out = s->tmp;
  for (int i = 0; i <= s->c.nx; i++)
    for (int k = 0; k <= s->c.nz; k++) {
      double v;
      if (hx && hz) v = 0.25 * (rd(s, F, i - 1, k - 1) + rd(s, F, i, k - 1) + rd(s, F, i - 1, k) + rd(s, F, i, k));
      else if (hx) v = 0.5 * (rd(s, F, i - 1, k) + rd(s, F, i, k));
      else if (hz) v = 0.5 * (rd(s, F, i, k - 1) + rd(s, F, i, k));
      else v = F[IDX(s, i, k)];
      out[IDX(s, i, k)] = v;
    }
  memcpy(F, out, sizeof(double) * s->ncell);
}

/* exported: apply the configured filter to a caller array of a component */
void orc_filter_field(orc_sim* s, int comp, double* F) { filter_component(s, comp, F); }

/* ------------------------------------------------------------------ */
/* Energy-conserving gather (Sec. 5): each component interpolated from its own
 * Yee location with the same shape order along every axis (PR-17). */
static void gather(const orc_sim* s, double x, double z, double* E, double* B) {
  int ord = s->c.order;
  double X = x / s->dx, Z = (z - s->z0) / s->dz;
  int fx = (int)floor(X), fz = (int)floor(Z);
  const double* src[6] = { s->fE[0], s->fE[1], s->fE[2], s->fB[0], s->fB[1], s->fB[2] };
  double out[6];
  for (int c = 0; c < 6; c++) {
    double acc = 0.0;
    for (int i = fx - 3; i <= fx + 3; i++) {
      double wx = orc_shape(ord, X - (i + (s->c.gather_nodal ? 0.0 : STX[c])));
      if (wx == 0.0) continue;
      for (int k = fz - 3; k <= fz + 3; k++) {
        double wz = orc_shape(ord, Z - (k + (s->c.gather_nodal ? 0.0 : STZ[c])));
        if (wz == 0.0) continue;
        acc += rd(s, src[c], i, k) * wx * wz;
      }
    }
    out[c] = acc;
  }
  E[0] = out[0]; E[1] = out[1]; E[2] = out[2];
  B[0] = out[3]; B[1] = out[4]; B[2] = out[5];
}

/* ------------------------------------------------------------------ */
/* Esirkepov charge-conserving deposition in 2D (Esirkepov 2001, cited in
 * Sec. 4.2.2) for one particle of charge*weight qw moving from (x0,z0) to
 * (x1,z1) during dt, with out-of-plane velocity vy. Nodes of rho at integer
 * cells; Jx at (i+1/2,k), Jz at (i,k+1/2), Jy at (i,k). The window is wider
 * than the support; shape values outside the support are zero. */
#define EW 9
static void esirkepov(orc_sim* s, double* Jx, double* Jy, double* Jz,
                      double x0, double z0, double x1, double z1, double vy, double qw) {
  int ord = s->c.order;
  double X0 = x0 / s->dx, Z0 = (z0 - s->z0) / s->dz;
  double X1 = x1 / s->dx, Z1 = (z1 - s->z0) / s->dz;
  int bx = (int)floor(X0 < X1 ? X0 : X1) - 3;
  int bz = (int)floor(Z0 < Z1 ? Z0 : Z1) - 3;
  double S0x[EW], S1x[EW], S0z[EW], S1z[EW], DSx[EW], DSz[EW];
  for (int a = 0; a < EW; a++) {
    S0x[a] = orc_shape(ord, X0 - (bx + a)); S1x[a] = orc_shape(ord, X1 - (bx + a));
    S0z[a] = orc_shape(ord, Z0 - (bz + a)); S1z[a] = orc_shape(ord, Z1 - (bz + a));
    DSx[a] = S1x[a] - S0x[a]; DSz[a] = S1z[a] - S0z[a];
  }
  double cx = -qw / (s->dz * s->dt);   /* Jx(i+1/2) - Jx(i-1/2) = cx * Wx(i) */
  double cz = -qw / (s->dx * s->dt);
  double cy = qw * vy / (s->dx * s->dz);
  /* Jx: prefix sum along x of Wx = DSx (S0z + DSz/2) */
  for (int b = 0; b < EW; b++) {
    double acc = 0.0;
    for (int a = 0; a < EW; a++) {
      acc += cx * DSx[a] * (S0z[b] + 0.5 * DSz[b]);
      int i = bx + a, k = bz + b;
      if (acc != 0.0 && i >= 0 && i <= s->c.nx && k >= 0 && k <= s->c.nz) Jx[IDX(s, i, k)] += acc;
    }
  }
  /* Jz: prefix sum along z of Wz = DSz (S0x + DSx/2) */
  for (int a = 0; a < EW; a++) {
    double acc = 0.0;
    for (int b = 0; b < EW; b++) {
      acc += cz * DSz[b] * (S0x[a] + 0.5 * DSx[a]);
      int i = bx + a, k = bz + b;
      if (acc != 0.0 && i >= 0 && i <= s->c.nx && k >= 0 && k <= s->c.nz) Jz[IDX(s, i, k)] += acc;
    }
  }
  /* Jy = qw vy Wy/(dx dz), Wy = S0x S0z + DSx S0z/2 + S0x DSz/2 + DSx DSz/3 */
  for (int a = 0; a < EW; a++)
    for (int b = 0; b < EW; b++) {
      double wy = S0x[a] * S0z[b] + 0.5 * DSx[a] * S0z[b] + 0.5 * S0x[a] * DSz[b] + DSx[a] * DSz[b] / 3.0;
      int i = bx + a, k = bz + b;
      if (wy != 0.0 && i >= 0 && i <= s->c.nx && k >= 0 && k <= s->c.nz) Jy[IDX(s, i, k)] += cy * wy;
    }
}

/* exported single-particle deposit into caller arrays (tests) */
void orc_deposit_one(orc_sim* s, double* Jx, double* Jy, double* Jz,
                     double x0, double z0, double x1, double z1, double vy, double qw) {
  esirkepov(s, Jx, Jy, Jz, x0, z0, x1, z1, vy, qw);
}

/* charge density of one particle at its position (same shape as the deposit) */
static void deposit_rho(const orc_sim* s, double* rho, double x, double z, double qw) {
  int ord = s->c.order;
  double X = x / s->dx, Z = (z - s->z0) / s->dz;
  int fx = (int)floor(X), fz = (int)floor(Z);
  for (int i = fx - 3; i <= fx + 3; i++)
    for (int k = fz - 3; k <= fz + 3; k++) {
      double w = orc_shape(ord, X - i) * orc_shape(ord, Z - k);
      if (w != 0.0 && i >= 0 && i <= s->c.nx && k >= 0 && k <= s->c.nz)
        rho[IDX(s, i, k)] += qw * w / (s->dx * s->dz);
    }
}

void orc_rho_one(orc_sim* s, double* rho, double x, double z, double qw) { deposit_rho(s, rho, x, z, qw); }

/* weights (macro-particle counts per unit length along y) of the test beam, in the order it was given */
void orc_beam_weights(orc_sim* s, const double* w) {
  orc_species* b = &s->sp[2];
  for (long j = 0; j < b->n; j++) b->w[j] = w[j];
}

/* ------------------------------------------------------------------ */
/* species storage */
static void sp_reserve(orc_species* p, long n) {
  if (n <= p->cap) return;
  long cap = p->cap ? p->cap : 1024;
  while (cap < n) cap *= 2;
#define RE(f, T) p->f = (T*)realloc(p->f, sizeof(T) * cap)
  RE(x, double); RE(z, double); RE(ux, double); RE(uy, double); RE(uz, double); RE(w, double);
  RE(id, uint32_t); RE(alive, int);
  RE(tc, double); RE(zf0, double); RE(uxb, double); RE(uyb, double); RE(uzb, double); RE(active, int);
  RE(zl, double);
#undef RE
  p->cap = cap;
}

static void sp_push(orc_species* p, double x, double z, double ux, double uy, double uz, double w, uint32_t id) {
  sp_reserve(p, p->n + 1);
  long j = p->n++;
  p->x[j] = x; p->z[j] = z; p->ux[j] = ux; p->uy[j] = uy; p->uz[j] = uz; p->w[j] = w;
  p->id[j] = id; p->alive[j] = 1;
  p->tc[j] = 0; p->zf0[j] = 0; p->uxb[j] = 0; p->uyb[j] = 0; p->uzb[j] = 0; p->active[j] = 1;
  p->zl[j] = 0;
}

static void sp_compact(orc_species* p) {
  long o = 0;
  for (long j = 0; j < p->n; j++) {
    if (!p->alive[j]) continue;
    if (o != j) {
      p->x[o] = p->x[j]; p->z[o] = p->z[j]; p->ux[o] = p->ux[j]; p->uy[o] = p->uy[j]; p->uz[o] = p->uz[j];
      p->w[o] = p->w[j]; p->id[o] = p->id[j]; p->alive[o] = 1;
      p->tc[o] = p->tc[j]; p->zf0[o] = p->zf0[j]; p->uxb[o] = p->uxb[j]; p->uyb[o] = p->uyb[j];
      p->uzb[o] = p->uzb[j]; p->active[o] = p->active[j]; p->zl[o] = p->zl[j];
    }
    o++;
  }
  p->n = o;
}

/* ------------------------------------------------------------------ */
static double time_of(const orc_sim* s, long n) { return (double)n * s->dt; }

orc_sim* orc_create(const orc_config* cfg) {
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->c = *cfg;
  s->gamma = cfg->gamma_boost < 1.0 ? 1.0 : cfg->gamma_boost;
  s->beta = sqrt(1.0 - 1.0 / (s->gamma * s->gamma));
  /* boosted longitudinal cell dz* = (1+beta) gamma dz_lab (Sec. 5.1.1) */
  s->dz = (1.0 + s->beta) * s->gamma * cfg->dz_lab;
  s->dx = cfg->dx;
  s->a2 = cfg->ck_alpha + 2.0 * cfg->ck_beta;
  s->b2 = cfg->ck_beta + 2.0 * cfg->ck_gamma;
  if (cfg->dt_override > 0.0) s->dt = cfg->dt_override;
  else s->dt = cfg->courant * orc_cfl_2d(cfg->ck_alpha, cfg->ck_beta, cfg->ck_gamma, s->dx, s->dz, cfg->theta);
  s->nxp = cfg->nx + 1; s->nzp = cfg->nz + 1;
  s->ncell = (long)s->nxp * s->nzp;
  for (int c = 0; c < ONCOMP; c++) s->F[c] = (double*)calloc(s->ncell, sizeof(double));
  for (int c = 0; c < 3; c++) {
    s->Ep[c] = (double*)calloc(s->ncell, sizeof(double));
    s->Eb[c] = (double*)calloc(s->ncell, sizeof(double));
    s->Ee[c] = (double*)calloc(s->ncell, sizeof(double));
    s->Bold[c] = (double*)calloc(s->ncell, sizeof(double));
    s->fE[c] = (double*)calloc(s->ncell, sizeof(double));
    s->fB[c] = (double*)calloc(s->ncell, sizeof(double));
  }
  s->Byx = (double*)calloc(s->ncell, sizeof(double)); s->Byz = (double*)calloc(s->ncell, sizeof(double));
  s->Eyx = (double*)calloc(s->ncell, sizeof(double)); s->Eyz = (double*)calloc(s->ncell, sizeof(double));
  s->tmp = (double*)calloc(s->ncell, sizeof(double));
  s->sx_int = (double*)calloc(s->nxp + 1, sizeof(double)); s->sx_half = (double*)calloc(s->nxp + 1, sizeof(double));
  s->sz_int = (double*)calloc(s->nzp + 1, sizeof(double)); s->sz_half = (double*)calloc(s->nzp + 1, sizeof(double));
  int px = !cfg->periodic_x, pz = !cfg->periodic_z;
  for (int i = 0; i <= cfg->nx; i++) {
    s->sx_int[i] = px ? pml_sigma(s, i, cfg->nx, s->dx) : 0.0;
    s->sx_half[i] = px ? pml_sigma(s, i + 0.5, cfg->nx, s->dx) : 0.0;
  }
  for (int k = 0; k <= cfg->nz; k++) {
    s->sz_int[k] = pz ? pml_sigma(s, k, cfg->nz, s->dz) : 0.0;
    s->sz_half[k] = pz ? pml_sigma(s, k + 0.5, cfg->nz, s->dz) : 0.0;
  }
  int g = cfg->particle_guard;
  if (g < 0) {
    int P = cfg->filter_passes + (cfg->filter_compensate ? 1 : 0);
    int ssum = cfg->filter_stride;
    if (cfg->filter_strides[0] > 0) {
      ssum = 0;
      for (int q = 0; q < 4 && cfg->filter_strides[q] > 0; q++) ssum += cfg->filter_strides[q];
    }
    g = (cfg->order == 3 ? 3 : 2) + P * ssum + 2;
  }
  s->c.particle_guard = g;
  int L = cfg->pml_cells > 0 ? cfg->pml_cells : 0;
  s->gx_lo = L + g; s->gx_hi = cfg->nx - L - g;
  s->gz_lo = L + g; s->gz_hi = cfg->nz - L - g;
  s->sp[0].q = -O_QE; s->sp[0].m = O_ME;
  s->sp[1].q = O_QE;  s->sp[1].m = 1836.15267343 * O_ME;
  s->sp[2].q = -O_QE; s->sp[2].m = O_ME;
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  for (int c = 0; c < ONCOMP; c++) free(s->F[c]);
  for (int c = 0; c < 3; c++) { free(s->Ep[c]); free(s->Eb[c]); free(s->Ee[c]); free(s->Bold[c]); free(s->fE[c]); free(s->fB[c]); }
  free(s->Byx); free(s->Byz); free(s->Eyx); free(s->Eyz); free(s->tmp);
  free(s->sx_int); free(s->sx_half); free(s->sz_int); free(s->sz_half);
  for (int j = 0; j < 3; j++) {
    orc_species* p = &s->sp[j];
    free(p->x); free(p->z); free(p->ux); free(p->uy); free(p->uz); free(p->w); free(p->id); free(p->alive);
    free(p->tc); free(p->zf0); free(p->uxb); free(p->uyb); free(p->uzb); free(p->active); free(p->zl);
  }
  free(s->rzL); free(s->rtL); free(s->rout); free(s->rdone);
  for (int c = 0; c < 3; c++) free(s->ext[c]);
  free(s->ext_prof);
  free(s);
}

/* info: dx, dz, dt, gamma, beta, z0, step, t, guard, gx_lo, gx_hi, gz_lo, gz_hi */
void orc_info(const orc_sim* s, double* out) {
  out[0] = s->dx; out[1] = s->dz; out[2] = s->dt; out[3] = s->gamma; out[4] = s->beta;
  out[5] = s->z0; out[6] = (double)s->step; out[7] = time_of(s, s->step);
  out[8] = s->c.particle_guard; out[9] = s->gx_lo; out[10] = s->gx_hi; out[11] = s->gz_lo; out[12] = s->gz_hi;
  out[13] = s->beam_vbar;
}

/* ------------------------------------------------------------------ */
/* Plasma input (Sec. 3.1.1, PR-9, PR-12): a cold plasma fixed in the lab, laid
 * on a regular lattice. In the computational frame (moving at beta c) the
 * lattice row m sits at z'_m(t) = (m + 1/2) h - beta c t with h = dz/ppc_z;
 * its lab position z_lab = gamma (m + 1/2) h is fixed, and its density is
 * n' = gamma n0(z_lab). With a moving window (lab frame) the same formulas
 * hold with gamma = 1. Macro-particle weight w = n' dx dz/(ppc_x ppc_z) (per
 * unit length along y). Rows enter through the plane z = z_hi. */
static double lab_density(const orc_plasma* p, double zl) {
  if (zl < p->z_start_lab) return 0.0;
  double r = zl - p->z_start_lab;
  if (p->ramp_lab > 0.0 && r < p->ramp_lab) return p->n0 * r / p->ramp_lab;
  double plateau_end = p->ramp_lab + p->length_lab;
  if (p->length_lab > 0.0 && r >= plateau_end) return 0.0;
  return p->n0;
}

static double z_hi_of(const orc_sim* s) { return s->z0 + s->gz_hi * s->dz; }
static double z_lo_of(const orc_sim* s) { return s->z0 + s->gz_lo * s->dz; }

/* first lattice row not yet inside the plane z_hi at time t: ceil((z_hi + beta c t)/h - 1/2) */
static long rows_inside(const orc_sim* s, double t) {
  double y = (z_hi_of(s) + s->beta * O_C * t) / s->h_row - 0.5;
  return (long)ceil(y);
}

static void add_row(orc_sim* s, long m, double t) {
  double zlat = (m + 0.5) * s->h_row;
  double zl = s->gamma * zlat;
  double n = s->gamma * lab_density(&s->pl, zl);
  if (n <= 0.0) return;
  double zp = zlat - s->beta * O_C * t;
  double w = n * s->dx * s->dz / (double)(s->pl.ppc_x * s->pl.ppc_z);
  double uz = -s->gamma * s->beta * O_C;
  for (long a = 0; a < s->nxl; a++) {
    double xp = (s->gx_lo + (a + 0.5) / s->pl.ppc_x) * s->dx;
    uint32_t id = (uint32_t)((uint64_t)m * (uint64_t)s->nxl + (uint64_t)a);
    sp_push(&s->sp[0], xp, zp, 0.0, 0.0, uz, w, id);
    if (s->pl.ions) {
      sp_push(&s->sp[1], xp, zp, 0.0, 0.0, uz, w, id);
      s->sp[1].zl[s->sp[1].n - 1] = zlat;
    }
  }
}

int orc_load_plasma(orc_sim* s, const orc_plasma* p) {
  s->pl = *p; s->has_plasma = 1;
  s->h_row = s->dz / p->ppc_z;
  s->nxl = (long)(s->gx_hi - s->gx_lo) * p->ppc_x;
  double t = time_of(s, s->step);
  long m_end = rows_inside(s, t);
  long m_beg = (long)ceil((z_lo_of(s) + s->beta * O_C * t) / s->h_row - 0.5);
  for (long m = m_beg; m < m_end; m++) add_row(s, m, t);
  s->row_next_e = m_end;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Laser input through a plane (Sec. 3.1.2). The lab waveform at the antenna is
 * g(x,s) = E0 exp(-(x-xc)^2/w0^2) exp(-(s-t_peak)^2/(2 sigma_t^2)) sin(omega (s - t_peak) + phase)
 * (PR-14). For a plane moving at beta_s in the computational frame the field
 * to emit is (1-beta_s) E'0 f sin((1-beta_s) omega' t'), E'0/E0 = omega'/omega
 * = 1/((1+beta) gamma) (Sec. 3.1.2), i.e. E_emit = (1-beta_s)/((1+beta) gamma)
 * g(x, (1-beta_s) t'/((1+beta) gamma)). The antenna is a sheet of +/- pairs
 * (one per transverse node) whose out-of-plane motion carries the surface
 * current K_y = -2 eps0 c E_emit (PR-13): only Jy is deposited in 2D. */
int orc_set_laser(orc_sim* s, const orc_laser* l) { s->las = *l; s->has_laser = 1; return 0; }

static double emit_field(const orc_sim* s, double x, double tp) {
  const orc_laser* l = &s->las;
  double om = 2.0 * O_PI * O_C / l->lambda0;
  double E0 = l->a0 * O_ME * O_C * om / O_QE;
  double dop = (1.0 + s->beta) * s->gamma;
  double sl = (1.0 - l->beta_s) * tp / dop;
  double sig = l->tau_fwhm / (2.0 * sqrt(log(2.0)));
  double dxr = x - l->x_center;
  double g = E0 * exp(-dxr * dxr / (l->w0 * l->w0)) * exp(-(sl - l->t_peak) * (sl - l->t_peak) / (2.0 * sig * sig))
             * sin(om * (sl - l->t_peak) + l->phase);
  return (1.0 - l->beta_s) / dop * g;
}

static void antenna(orc_sim* s) {
  if (!s->has_laser) return;
  int ord = s->c.order;
  double t0 = time_of(s, s->step), t1 = time_of(s, s->step + 1), th = 0.5 * (t0 + t1);
  double za0 = s->las.z_antenna + s->las.beta_s * O_C * t0;
  double za1 = s->las.z_antenna + s->las.beta_s * O_C * t1;
  double zlo = z_lo_of(s), zhi = z_hi_of(s);
  if (za0 < zlo || za0 >= zhi || za1 < zlo || za1 >= zhi) return;
  double Z0 = (za0 - s->z0) / s->dz, Z1 = (za1 - s->z0) / s->dz;
  int fz = (int)floor(Z0 < Z1 ? Z0 : Z1);
  double* Jy = s->F[OJY];
  for (int ia = s->gx_lo; ia <= s->gx_hi; ia++) {
    double K = -2.0 * O_EPS0 * O_C * emit_field(s, ia * s->dx, th);
    if (K == 0.0) continue;
    for (int i = ia - 2; i <= ia + 2; i++) {
      double wx = orc_shape(ord, (double)(ia - i));
      if (wx == 0.0) continue;
      for (int k = fz - 3; k <= fz + 4; k++) {
        double wz = 0.5 * (orc_shape(ord, Z0 - k) + orc_shape(ord, Z1 - k));
        if (wz == 0.0 || i < 0 || i > s->c.nx || k < 0 || k > s->c.nz) continue;
        Jy[IDX(s, i, k)] += K * wx * wz / s->dz;
      }
    }
  }
}

/* ------------------------------------------------------------------ */
/* Test beam through a plane (Sec. 3.1.1, Eq. t*..Eq. zp): lab particles given
 * at lab time t_lab are projected ballistically onto the lab plane z_plane,
 * Lorentz-transformed to the computational frame (velocities with the mean
 * beam velocity beta_b, Eq. vxp*..vzp*) and synchronised to t' = 0 with the
 * mean boosted velocity; they stay frozen until t' reaches their crossing
 * time, then become active test particles (gather + push, no deposit). */
int orc_set_beam(orc_sim* s, long n, const double* x, const double* z, const double* ux,
                 const double* uy, const double* uz, double t_lab, double z_plane) {
  orc_species* b = &s->sp[2];
  double g = s->gamma, be = s->beta;
  double vzsum = 0.0;
  for (long j = 0; j < n; j++) {
    double gj = sqrt(1.0 + (ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) / (O_C * O_C));
    vzsum += uz[j] / gj;
  }
  double betab = vzsum / n / O_C;
  double vpsum = 0.0;
  double* tcv = (double*)malloc(sizeof(double) * n);
  double* zcv = (double*)malloc(sizeof(double) * n);
  for (long j = 0; j < n; j++) {
    double gj = sqrt(1.0 + (ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) / (O_C * O_C));
    double vx = ux[j] / gj, vy = uy[j] / gj, vz = uz[j] / gj;
    double tcross = t_lab + (z_plane - z[j]) / vz;          /* ballistic projection onto the plane */
    double xs = x[j] + vx * (tcross - t_lab);
    double tpc = g * (tcross - be * z_plane / O_C);          /* crossing event in the boosted frame */
    double zpc = g * (z_plane - be * O_C * tcross);
    double den = 1.0 - be * betab;
    double vxp = vx / (g * den), vyp = vy / (g * den), vzp = (vz - be * O_C) / den;
    vpsum += vzp;
    double v2 = (vxp * vxp + vyp * vyp + vzp * vzp) / (O_C * O_C);
    double gp = 1.0 / sqrt(1.0 - v2);
    sp_push(b, xs, 0.0, gp * vxp, gp * vyp, gp * vzp, 1.0, (uint32_t)j);
    tcv[j] = tpc; zcv[j] = zpc;
  }
  double vbar = vpsum / n;
  for (long j = 0; j < n; j++) {
    long q = b->n - n + j;
    b->tc[q] = tcv[j];
    b->zf0[q] = zcv[j] - vbar * tcv[j];                      /* synchronised position at t' = 0 */
    b->uxb[q] = b->ux[q]; b->uyb[q] = b->uy[q]; b->uzb[q] = b->uz[q];
    b->active[q] = 0;
    b->z[q] = b->zf0[q] + vbar * time_of(s, s->step);
  }
  free(tcv); free(zcv);
  s->beam_vbar = vbar; s->has_beam = 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* back-transformed diagnostics (Sec. 3.2, PR-16): a lab sample row (z_L, t_L)
 * maps to t' = gamma (t_L - beta z_L/c), z' = gamma (z_L - beta c t_L); E is
 * linearly interpolated between E^n and E^{n+1} (t' in [t^n, t^{n+1})), B
 * between B^{n-1/2} and B^{n+1/2}, both linearly in z' on their own mesh,
 * then transformed to the lab. Each row stores 6 components x (nx+1). */
int orc_btd_set(orc_sim* s, int nrows, const double* zL, const double* tL) {
  free(s->rzL); free(s->rtL); free(s->rout); free(s->rdone);
  s->nrows = nrows;
  s->rzL = (double*)malloc(sizeof(double) * nrows); s->rtL = (double*)malloc(sizeof(double) * nrows);
  memcpy(s->rzL, zL, sizeof(double) * nrows); memcpy(s->rtL, tL, sizeof(double) * nrows);
  s->rout = (double*)calloc((size_t)nrows * 6 * s->nxp, sizeof(double));
  s->rdone = (int*)calloc((size_t)nrows * 2, sizeof(int));
  return 0;
}

static double interp_z(const orc_sim* s, const double* F, int i, double zp, double stz) {
  double Z = (zp - s->z0) / s->dz - stz;
  int k = (int)floor(Z);
  double f = Z - k;
  return (1.0 - f) * rd(s, F, i, k) + f * rd(s, F, i, k + 1);
}

/* which = 0: E-part with fields E (weight we); which = 1: B-part */
static void btd_accumulate(orc_sim* s, int which, int post) {
  double g = s->gamma, be = s->beta;
  for (int r = 0; r < s->nrows; r++) {
    double tp = g * (s->rtL[r] - be * s->rzL[r] / O_C);
    double zp = g * (s->rzL[r] - be * O_C * s->rtL[r]);
    double ta, tb;
    if (which == 0) { ta = time_of(s, s->step); tb = time_of(s, s->step + 1); }
    else { ta = time_of(s, s->step) - 0.5 * s->dt; tb = ta + s->dt; }
    if (!(tp >= ta && tp < tb)) continue;
    double f = (tp - ta) / s->dt;
    double wgt = post ? f : 1.0 - f;
    double* out = s->rout + (size_t)r * 6 * s->nxp;
    for (int i = 0; i <= s->c.nx; i++) {
      if (which == 0) {
        double ex = interp_z(s, s->F[OEX], i, zp, STZ[OEX]);
        double ey = interp_z(s, s->F[OEY], i, zp, STZ[OEY]);
        double ez = interp_z(s, s->F[OEZ], i, zp, STZ[OEZ]);
        out[0 * s->nxp + i] += wgt * g * ex;          /* Ex_lab = g (Ex' + beta c By') */
        out[1 * s->nxp + i] += wgt * g * ey;          /* Ey_lab = g (Ey' - beta c Bx') */
        out[2 * s->nxp + i] += wgt * ez;
        out[3 * s->nxp + i] += wgt * (-g * be * ey / O_C); /* Bx_lab = g (Bx' - beta Ey'/c) */
        out[4 * s->nxp + i] += wgt * (g * be * ex / O_C);  /* By_lab = g (By' + beta Ex'/c) */
      } else {
        double bx = interp_z(s, s->F[OBX], i, zp, STZ[OBX]);
        double by = interp_z(s, s->F[OBY], i, zp, STZ[OBY]);
        double bz = interp_z(s, s->F[OBZ], i, zp, STZ[OBZ]);
        out[0 * s->nxp + i] += wgt * g * be * O_C * by;
        out[1 * s->nxp + i] += wgt * (-g * be * O_C * bx);
        out[3 * s->nxp + i] += wgt * g * bx;
        out[4 * s->nxp + i] += wgt * g * by;
        out[5 * s->nxp + i] += wgt * bz;
      }
    }
    if (post) s->rdone[2 * r + which] = 1;
  }
}

int orc_btd_get(const orc_sim* s, double* out, int* done) {
  memcpy(out, s->rout, sizeof(double) * (size_t)s->nrows * 6 * s->nxp);
  memcpy(done, s->rdone, sizeof(int) * (size_t)s->nrows * 2);
  return 0;
}

/* ------------------------------------------------------------------ */
/* moving window (Sec. 2: lab-frame runs follow the wake): the grid moves by
 * whole cells; fields are shifted toward -z and zero-filled at +z. */
static void shift_array(orc_sim* s, double* F, long sh, int comp) {
  int i0, i1, k0, k1;
  vrange(s, comp, &i0, &i1, &k0, &k1);
  for (int i = 0; i <= s->c.nx; i++)
    for (int k = 0; k <= s->c.nz; k++) {
      long kk = k + sh;
      double v = kk <= s->c.nz ? F[IDX(s, i, (int)kk)] : 0.0;
      /* the PEC walls move with the grid: values stay on the component's valid range */
      F[IDX(s, i, k)] = (i >= i0 && i <= i1 && k >= k0 && k <= k1) ? v : 0.0;
    }
}

static void window_shift(orc_sim* s) {
  if (!s->c.moving_window) return;
  double t = time_of(s, s->step);
  long want = (long)floor(s->c.window_beta * O_C * t / s->dz);
  long sh = want - s->shifts;
  if (sh <= 0) return;
  for (int c = 0; c < 6; c++) shift_array(s, s->F[c], sh, c);
  for (int c = 0; c < 3; c++) { shift_array(s, s->Ep[c], sh, c); shift_array(s, s->Eb[c], sh, c); }
  shift_array(s, s->Byx, sh, OBY); shift_array(s, s->Byz, sh, OBY);
  shift_array(s, s->Eyx, sh, OEY); shift_array(s, s->Eyz, sh, OEY);
  s->shifts = want;
  s->z0 = want * s->dz;
}

/* ------------------------------------------------------------------ */
/* One PIC step in the order of PR-1. */
static void one_step(orc_sim* s) {
  window_shift(s);
  btd_accumulate(s, 0, 0);
  btd_accumulate(s, 1, 0);
  /* 1. Faraday + Friedman + PML-B */
  faraday(s);
  /* 2. gather copies: E^n and B^n = (B^{n-1/2} + B^{n+1/2})/2, filtered (Sec. 4: gathered fields) */
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < s->ncell; p++) {
      s->fE[c][p] = s->F[OEX + c][p];
      s->fB[c][p] = 0.5 * (s->Bold[c][p] + s->F[OBX + c][p]);
    }
  if (s->c.filter_gather) {
    for (int c = 0; c < 3; c++) { filter_component(s, OEX + c, s->fE[c]); filter_component(s, OBX + c, s->fB[c]); }
  }
  if (s->c.gather_nodal)
    for (int c = 0; c < 3; c++) { to_nodes(s, OEX + c, s->fE[c]); to_nodes(s, OBX + c, s->fB[c]); }
  /* 3-5. particles: gather, Boris, move, Esirkepov */
  for (int c = OJX; c <= OJZ; c++) memset(s->F[c], 0, sizeof(double) * s->ncell);
  double xlo = s->gx_lo * s->dx, xhi = s->gx_hi * s->dx;
  double zlo = z_lo_of(s), zhi = z_hi_of(s) + s->dz;
  double tn = time_of(s, s->step), tn1 = time_of(s, s->step + 1);
  for (int j = 0; j < 3; j++) {
    orc_species* p = &s->sp[j];
    for (long q = 0; q < p->n; q++) {
      if (!p->alive[q]) continue;
      if (j == 2 && !p->active[q]) {
        if (tn >= p->tc[q]) {
          p->active[q] = 1;
          p->ux[q] = p->uxb[q]; p->uy[q] = p->uyb[q]; p->uz[q] = p->uzb[q];
          /* a particle whose crossing lies outside the particle domain never enters it (PR-20) */
          if (p->x[q] < xlo || p->x[q] >= xhi || p->z[q] < zlo || p->z[q] >= zhi) { p->alive[q] = 0; continue; }
        } else {
          const double zn = p->zf0[q] + s->beam_vbar * tn1;
          /* a frozen particle inside the particle domain carries its charge along z at the mean velocity */
          if (s->c.beam_self && p->x[q] >= xlo && p->x[q] < xhi && p->z[q] >= zlo && p->z[q] < zhi && zn >= zlo &&
              zn < zhi)
            esirkepov(s, s->F[OJX], s->F[OJY], s->F[OJZ], p->x[q], p->z[q], p->x[q], zn, 0.0, p->q * p->w[q]);
          p->z[q] = zn;
          continue;
        }
      }
      double u[3] = { p->ux[q], p->uy[q], p->uz[q] };
      if (j != 1) {
        double E[3], B[3];
        gather(s, p->x[q], p->z[q], E, B);
        orc_boris(u, E, B, p->q, p->m, s->dt);
      }
      double gm = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (O_C * O_C));
      double xn = p->x[q] + s->dt * u[0] / gm;
      double zn = p->z[q] + s->dt * u[2] / gm;
      if (j == 1) {
        /* ions are fixed in the lab: they stay on z'(t) = (m + 1/2) h - beta c t (PR-9, PR-12) */
        xn = p->x[q];
        p->z[q] = p->zl[q] - s->beta * O_C * tn;
        zn = p->zl[q] - s->beta * O_C * tn1;
      }
      if (j != 2 || s->c.beam_self)
        esirkepov(s, s->F[OJX], s->F[OJY], s->F[OJZ], p->x[q], p->z[q], xn, zn, u[1] / gm, p->q * p->w[q]);
      p->x[q] = xn; p->z[q] = zn; p->ux[q] = u[0]; p->uy[q] = u[1]; p->uz[q] = u[2];
      if (xn < xlo || xn >= xhi || zn < zlo || zn >= zhi) p->alive[q] = 0;
    }
  }
  /* 6. antenna current, external test source */
  antenna(s);
  for (int c = 0; c < 3; c++)
    if (s->ext[c]) {
      double sg = (s->ext_alternate && (s->step & 1)) ? -1.0 : 1.0;
      if (s->ext_prof) sg *= s->step < s->ext_nprof ? s->ext_prof[s->step] : 0.0;
      for (long p = 0; p < s->ncell; p++) s->F[OJX + c][p] += sg * s->ext[c][p];
    }
  /* 7. current filter */
  if (s->c.filter_J) for (int c = 0; c < 3; c++) filter_component(s, OJX + c, s->F[OJX + c]);
  /* 8. Ampere + PML-E */
  ampere(s);
  btd_accumulate(s, 0, 1);
  btd_accumulate(s, 1, 1);
  /* 9. particle removal and inflow through the plane z_hi */
  sp_compact(&s->sp[0]); sp_compact(&s->sp[1]);
  if (s->has_plasma) {
    long m_end = rows_inside(s, tn1);
    for (long m = s->row_next_e; m < m_end; m++) add_row(s, m, tn1);
    if (m_end > s->row_next_e) s->row_next_e = m_end;
  }
  s->step++;
}

int orc_step(orc_sim* s, int n) {
  for (int i = 0; i < n; i++) one_step(s);
  return 0;
}

/* ------------------------------------------------------------------ */
/* accessors */
void orc_get_field(const orc_sim* s, int comp, double* out) { memcpy(out, s->F[comp], sizeof(double) * s->ncell); }
void orc_set_field(orc_sim* s, int comp, const double* in) { memcpy(s->F[comp], in, sizeof(double) * s->ncell); }
void orc_get_gather_field(const orc_sim* s, int comp, double* out) {
  memcpy(out, comp < 3 ? s->fE[comp] : s->fB[comp - 3], sizeof(double) * s->ncell);
}
/* Friedman history: which = 0 E^{n-1}, 1 E-bar */
void orc_get_history(const orc_sim* s, int which, int comp, double* out) {
  memcpy(out, which == 0 ? s->Ep[comp] : s->Eb[comp], sizeof(double) * s->ncell);
}
void orc_set_history(orc_sim* s, int which, int comp, const double* in) {
  memcpy(which == 0 ? s->Ep[comp] : s->Eb[comp], in, sizeof(double) * s->ncell);
}
/* external current J_comp (A/m^2) added every step before the current filter;
 * alternate != 0 flips its sign on odd steps (source modulated at the Nyquist frequency) */
void orc_set_ext_current(orc_sim* s, int comp, const double* in, int alternate) {
  if (!s->ext[comp]) s->ext[comp] = (double*)malloc(sizeof(double) * s->ncell);
  memcpy(s->ext[comp], in, sizeof(double) * s->ncell);
  s->ext_alternate = alternate;
}
/* optional per-step multiplier of the external current (0 after the table ends) */
void orc_set_ext_profile(orc_sim* s, long n, const double* prof) {
  free(s->ext_prof);
  s->ext_prof = (double*)malloc(sizeof(double) * (n > 0 ? n : 1));
  memcpy(s->ext_prof, prof, sizeof(double) * n);
  s->ext_nprof = n;
}
long orc_num_particles(const orc_sim* s, int species) { return s->sp[species].n; }
void orc_get_particles(const orc_sim* s, int species, double* x, double* z, double* ux, double* uy,
                       double* uz, double* w, uint32_t* id, int* flag) {
  const orc_species* p = &s->sp[species];
  for (long j = 0; j < p->n; j++) {
    x[j] = p->x[j]; z[j] = p->z[j]; ux[j] = p->ux[j]; uy[j] = p->uy[j]; uz[j] = p->uz[j];
    w[j] = p->w[j]; id[j] = p->id[j]; flag[j] = (p->alive[j] ? 1 : 0) | (p->active[j] ? 2 : 0);
  }
}
void orc_set_particles(orc_sim* s, int species, long n, const double* x, const double* z, const double* ux,
                       const double* uy, const double* uz, const double* w) {
  orc_species* p = &s->sp[species];
  p->n = 0;
  for (long j = 0; j < n; j++) sp_push(p, x[j], z[j], ux[j], uy[j], uz[j], w[j], (uint32_t)j);
}

/* total charge density of all depositing species at their current positions */
void orc_rho(const orc_sim* s, double* rho) {
  memset(rho, 0, sizeof(double) * s->ncell);
  for (int j = 0; j < 2; j++) {
    const orc_species* p = &s->sp[j];
    for (long q = 0; q < p->n; q++)
      if (p->alive[q]) deposit_rho(s, rho, p->x[q], p->z[q], p->q * p->w[q]);
  }
}

/* diagnostics (Sec. 5, Fig. energy/time histories): out = [n_e, n_beam_active,
 * <gamma_lab> of active beam, rms(gamma_lab)/<gamma_lab>, field energy per unit y] */
void orc_diag(const orc_sim* s, double* out) {
  const orc_species* b = &s->sp[2];
  double sum = 0.0, sum2 = 0.0; long na = 0;
  for (long j = 0; j < b->n; j++) {
    if (!b->alive[j] || !b->active[j]) continue;
    double gp = sqrt(1.0 + (b->ux[j] * b->ux[j] + b->uy[j] * b->uy[j] + b->uz[j] * b->uz[j]) / (O_C * O_C));
    double gl = s->gamma * (gp + s->beta * b->uz[j] / O_C);
    sum += gl; sum2 += gl * gl; na++;
  }
  double mean = na ? sum / na : 0.0;
  double var = na ? sum2 / na - mean * mean : 0.0;
  double en = 0.0;
  for (long p = 0; p < s->ncell; p++) {
    double e2 = s->F[OEX][p] * s->F[OEX][p] + s->F[OEY][p] * s->F[OEY][p] + s->F[OEZ][p] * s->F[OEZ][p];
    double b2 = s->F[OBX][p] * s->F[OBX][p] + s->F[OBY][p] * s->F[OBY][p] + s->F[OBZ][p] * s->F[OBZ][p];
    en += 0.5 * (O_EPS0 * e2 + b2 / O_MU0) * s->dx * s->dz;
  }
  out[0] = (double)s->sp[0].n; out[1] = (double)na; out[2] = mean;
  out[3] = mean > 0 ? sqrt(var > 0 ? var : 0) / mean : 0.0; out[4] = en;
}
