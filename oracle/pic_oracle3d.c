/*
 * FP64 CPU oracle of the boosted-frame electromagnetic PIC step in 3D (x,y,z).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library. The product
 * path (the CUDA library behind include/pic.h) neither links nor calls it, and
 * this file includes no header of the product.
 *
 * Same method as the 2-1/2D oracle (pic_oracle.c), written out in three
 * dimensions from the paper (Vay et al., arXiv:1009.2727):
 *   - Sec. 4.2  Faraday with the enlarged operator Delta*_x = (alpha + beta S1_x
 *               + gamma S2_x) Delta_x, S1 and S2 sums of the transverse
 *               neighbours one full cell away (PR-2), Ampere with the Yee operator;
 *   - Sec. 4.3  Friedman damping (Eq. Faraday_Friedman);
 *   - Sec. 4.1  bilinear filter passes + compensation along x, then y, then z;
 *   - App. II   split-field PML on all six faces: every component is the sum
 *               of two parts, one per derivative direction;
 *   - Sec. 4.2.2 Esirkepov deposition in 3D (Esirkepov 2001);
 *   - Sec. 5    cubic (or linear) B-spline shapes, energy-conserving gather;
 *   - Sec. 3.1  plasma and test beam through planes; the laser from two dual
 *               arrays of macro-particles, one pair per transverse cell of the
 *               antenna plane: the moving partner is displaced along y (the
 *               polarisation) and deposits with Esirkepov, so Gauss's law holds;
 *   - Sec. 3.2  lab-frame samples by interpolation, one transverse slice per row.
 * Boris push: the textbook scheme (orc_boris of pic_oracle.c, same library).
 *
 * Layout: node (i,j,k) of every (nx+1)(ny+1)(nz+1) array at (i*(ny+1)+j)*(nz+1)+k.
 * Yee positions: Ex (i+1/2,j,k), Ey (i,j+1/2,k), Ez (i,j,k+1/2),
 * Bx (i,j+1/2,k+1/2), By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k); J like E.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define O_C 299792458.0
#define O_QE 1.602176634e-19
#define O_ME 9.1093837015e-31
#define O_EPS0 8.8541878128e-12
#define O_MU0 (1.0 / (O_EPS0 * O_C * O_C))
#define O_PI 3.14159265358979323846

double orc_shape(int order, double s);
double orc_cfl_3d(double a, double b, double g, double dx, double dy, double dz, double theta);
void orc_boris(double* u, const double* E, const double* B, double q, double m, double dt);

enum { QEX = 0, QEY, QEZ, QBX, QBY, QBZ, QJX, QJY, QJZ, QNCOMP };

typedef struct {
  int nx, ny, nz;
  double dz_lab, dx, dy;
  double gamma_boost, courant, dt_override;
  double ck_alpha, ck_beta, ck_gamma, theta;
  int pml_cells;
  double pml_sigma_max, pml_delta, pml_power;
  int pml_xi_exp;
  int filter_passes, filter_stride, filter_compensate, filter_J, filter_gather;
  int order, particle_guard;
  int periodic_x, periodic_y, periodic_z;   /* fields only (test option) */
  int filter_strides[4];      /* > 0: product over these strides of (n passes + compensation), Sec. 4.1 */
  int gather_nodal;           /* 1: 'momentum conserving' gather from node-interpolated fields (Sec. 5) */
  int beam_self;              /* 1: the test beam's frozen and active particles deposit their current (Sec. 3.1.1) */
} o3_config;

typedef struct {
  double n0, z_start_lab, ramp_lab, length_lab;
  int ppc_x, ppc_y, ppc_z, ions;
} o3_plasma;

typedef struct {
  double lambda0, a0, w0, tau_fwhm, t_peak, x_center, y_center, phase, z_antenna;
} o3_laser;

typedef struct {
  double *x, *y, *z, *ux, *uy, *uz, *w;
  uint32_t* id;
  int* alive;
  double *tc, *zf0, *uxb, *uyb, *uzb; int* active;   /* test beam */
  double* zl;                                         /* ions: lattice position of the row */
  long n, cap;
  double q, m;
} o3_species;

typedef struct {
  o3_config c;
  double dx, dy, dz, dt, gamma, beta;
  int nxp, nyp, nzp;
  long ncell;
  double* F[QNCOMP];
  double *Ep[3], *Eb[3], *Ee[3], *Bold[3], *fE[3], *fB[3];
  double* Es[3][2];          /* split parts of E: Ex = (x,y)+(x,z), Ey = (y,z)+(y,x), Ez = (z,x)+(z,y) */
  double* Bs[3][2];          /* split parts of B in the same order */
  double* tmp;
  double *s_int[3], *s_half[3];   /* sigma at integer / half positions per axis */
  long step;
  int glo[3], ghi[3];        /* particle domain in cells per axis */
  o3_species sp[3];          /* 0 electrons, 1 ions, 2 test beam */
  o3_plasma pl; int has_plasma;
  long row_next, nxl, nyl;
  double h_row;
  o3_laser las; int has_laser;
  double q_pair;             /* charge of each antenna partner */
  double* delta;             /* antenna partner displacement along y per transverse node */
  double beam_vbar; int has_beam;
  int nrows; double *rzL, *rtL, *rout; int* rdone;
} o3_sim;

/* ------------------------------------------------------------------ */
static const double SX[QNCOMP] = { 0.5, 0.0, 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0 };
static const double SY[QNCOMP] = { 0.0, 0.5, 0.0, 0.5, 0.0, 0.5, 0.0, 0.5, 0.0 };
static const double SZ[QNCOMP] = { 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 0.5 };

static inline long I3(const o3_sim* s, int i, int j, int k) { return ((long)i * s->nyp + j) * s->nzp + k; }

static int wrap(int v, int n, int periodic) {
  if (!periodic) return v;
  v %= n;
  return v < 0 ? v + n : v;
}

static double rd(const o3_sim* s, const double* F, int i, int j, int k) {
  i = wrap(i, s->c.nx, s->c.periodic_x);
  j = wrap(j, s->c.ny, s->c.periodic_y);
  k = wrap(k, s->c.nz, s->c.periodic_z);
  if (i < 0 || i > s->c.nx || j < 0 || j > s->c.ny || k < 0 || k > s->c.nz) return 0.0;
  return F[I3(s, i, j, k)];
}

/* valid index range along one axis: a half-staggered index runs 0..n-1; an integer index runs 1..n-1
 * for E (tangential E vanishes on the PEC walls) and 0..n for B; periodic axes run 0..n-1 */
static void axis_range(const o3_sim* s, int comp, int axis, int* lo, int* hi) {
  int c = comp >= QJX ? comp - QJX : comp;
  const double* st = axis == 0 ? SX : axis == 1 ? SY : SZ;
  int n = axis == 0 ? s->c.nx : axis == 1 ? s->c.ny : s->c.nz;
  int per = axis == 0 ? s->c.periodic_x : axis == 1 ? s->c.periodic_y : s->c.periodic_z;
  if (per) { *lo = 0; *hi = n - 1; return; }
  if (st[c] > 0.0) { *lo = 0; *hi = n - 1; }
  else if (c < 3) { *lo = 1; *hi = n - 1; }
  else { *lo = 0; *hi = n; }
}

static double pml_sigma(const o3_sim* s, double pos, int n, double d_cell) {
  int L = s->c.pml_cells;
  if (L <= 0) return 0.0;
  double d = 0.0;
  if (pos < L) d = L - pos;
  if (pos > n - L) d = pos - (n - L);
  if (d <= 0.0) return 0.0;
  return s->c.pml_sigma_max * O_C / d_cell * pow(d / s->c.pml_delta, s->c.pml_power);
}

static double pml_xi(const o3_sim* s, double sig) {
  if (s->c.pml_xi_exp) return exp(-sig * s->dt);
  return (1.0 - 0.5 * sig * s->dt) / (1.0 + 0.5 * sig * s->dt);
}

static double pml_coef(const o3_sim* s, double sig) {
  if (sig <= 0.0) return s->dt;
  return (1.0 - pml_xi(s, sig)) / sig;
}

/* ------------------------------------------------------------------ */
/* Enlarged difference of F along axis a (Sec. 4.2, PR-2): with D(o1,o2) the plain difference
 * F(p + e_a + o1 e_b + o2 e_c) - F(p + o1 e_b + o2 e_c) over the two other axes b < c,
 * Delta*_a F = [alpha D(0,0) + beta (D(+-1,0) + D(0,+-1)) + gamma D(+-1,+-1)] / d_a.
 * The result sits half a cell above p along a. */
static double dstar(const o3_sim* s, const double* F, int a, int i, int j, int k) {
  int e[3][3] = { { 1, 0, 0 }, { 0, 1, 0 }, { 0, 0, 1 } };
  int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  double D[3][3];
  for (int o1 = -1; o1 <= 1; o1++)
    for (int o2 = -1; o2 <= 1; o2++) {
      int pi = i + o1 * e[b][0] + o2 * e[c][0];
      int pj = j + o1 * e[b][1] + o2 * e[c][1];
      int pk = k + o1 * e[b][2] + o2 * e[c][2];
      D[o1 + 1][o2 + 1] = rd(s, F, pi + e[a][0], pj + e[a][1], pk + e[a][2]) - rd(s, F, pi, pj, pk);
    }
  double sum1 = D[0][1] + D[2][1] + D[1][0] + D[1][2];
  double sum2 = D[0][0] + D[0][2] + D[2][0] + D[2][2];
  double d = a == 0 ? s->dx : a == 1 ? s->dy : s->dz;
  return (s->c.ck_alpha * D[1][1] + s->c.ck_beta * sum1 + s->c.ck_gamma * sum2) / d;
}

/* plain backward difference of F along axis a (Yee, Eq. Ampere): F(p) - F(p - e_a) */
static double dback(const o3_sim* s, const double* F, int a, int i, int j, int k) {
  double d = a == 0 ? s->dx : a == 1 ? s->dy : s->dz;
  double m = rd(s, F, i - (a == 0), j - (a == 1), k - (a == 2));
  return (rd(s, F, i, j, k) - m) / d;
}

static double sig_at(const o3_sim* s, int axis, int idx, int half) {
  return half ? s->s_half[axis][idx] : s->s_int[axis][idx];
}

/* ------------------------------------------------------------------ */
/* Faraday (Eq. Faraday) with the Friedman E_eff (Eq. Faraday_Friedman, PR-1) and the split-field PML:
 * dB_q/dt = -(Delta*_u E_v - Delta*_v E_u) for (q,u,v) cyclic; the part driven by the derivative along
 * an axis is damped by that axis' sigma at the component's position. */
static void faraday(o3_sim* s) {
  double th = s->c.theta;
  long N = s->ncell;
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < N; p++)
      s->Ee[c][p] = (1.0 + th / 4.0) * s->F[QEX + c][p] - 0.5 * s->Ep[c][p] + (0.5 - th / 4.0) * s->Eb[c][p];
  for (int c = 0; c < 3; c++) memcpy(s->Bold[c], s->F[QBX + c], sizeof(double) * N);
  for (int q = 0; q < 3; q++) {
    int u = (q + 1) % 3, v = (q + 2) % 3;    /* B_q -= dt (Delta*_u E_v - Delta*_v E_u) */
    int comp = QBX + q;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) axis_range(s, comp, a, &lo[a], &hi[a]);
    double* Bq = s->F[comp];
    /* split parts: [0] driven along u, [1] along v; the B_q position is half-staggered along u and v */
    double *Pu = s->Bs[q][0], *Pv = s->Bs[q][1];
    for (int i = lo[0]; i <= hi[0]; i++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int k = lo[2]; k <= hi[2]; k++) {
          int idx[3] = { i, j, k };
          double du = dstar(s, s->Ee[v], u, i, j, k);
          double dv = dstar(s, s->Ee[u], v, i, j, k);
          double su = sig_at(s, u, idx[u], 1), sv = sig_at(s, v, idx[v], 1);
          long p = I3(s, i, j, k);
          if (su > 0.0 || sv > 0.0) {
            Pu[p] = pml_xi(s, su) * Pu[p] - pml_coef(s, su) * du;
            Pv[p] = pml_xi(s, sv) * Pv[p] + pml_coef(s, sv) * dv;
            Bq[p] = Pu[p] + Pv[p];
          } else {
            Bq[p] = Bq[p] - s->dt * (du - dv);
          }
        }
  }
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < N; p++) {
      s->Eb[c][p] = (1.0 - th / 2.0) * s->F[QEX + c][p] + (th / 2.0) * s->Eb[c][p];
      s->Ep[c][p] = s->F[QEX + c][p];
    }
}

/* Ampere with the Yee operator (Eq. Ampere) and the split-field PML for E:
 * dE_q/dt = c^2 (Delta_u B_v - Delta_v B_u) - J_q/eps0; no current inside the PML (particle guard). */
static void ampere(o3_sim* s) {
  const double c2 = O_C * O_C;
  for (int q = 0; q < 3; q++) {
    int u = (q + 1) % 3, v = (q + 2) % 3;
    int comp = QEX + q;
    int lo[3], hi[3];
    for (int a = 0; a < 3; a++) axis_range(s, comp, a, &lo[a], &hi[a]);
    double* Eq = s->F[comp];
    const double* Jq = s->F[QJX + q];
    double *Pu = s->Es[q][0], *Pv = s->Es[q][1];
    for (int i = lo[0]; i <= hi[0]; i++)
      for (int j = lo[1]; j <= hi[1]; j++)
        for (int k = lo[2]; k <= hi[2]; k++) {
          int idx[3] = { i, j, k };
          double du = dback(s, s->F[QBX + v], u, i, j, k);
          double dv = dback(s, s->F[QBX + u], v, i, j, k);
          double su = sig_at(s, u, idx[u], 0), sv = sig_at(s, v, idx[v], 0);
          long p = I3(s, i, j, k);
          if (su > 0.0 || sv > 0.0) {
            Pu[p] = pml_xi(s, su) * Pu[p] + c2 * pml_coef(s, su) * du;
            Pv[p] = pml_xi(s, sv) * Pv[p] - c2 * pml_coef(s, sv) * dv;
            Eq[p] = Pu[p] + Pv[p];
          } else {
            Eq[p] = Eq[p] + s->dt * (c2 * (du - dv) - Jq[p] / O_EPS0);
          }
        }
  }
}

/* ------------------------------------------------------------------ */
/* Filter (Sec. 4.1): n bilinear passes (alpha 1/2) then the compensation pass (alpha_c = n/2 + 1),
 * along x, then y, then z; zero outside the component's valid range. */
static void filter_pass_axis(o3_sim* s, int comp, double* F, int axis, int stride, double alpha) {
  int lo[3], hi[3];
  for (int a = 0; a < 3; a++) axis_range(s, comp, a, &lo[a], &hi[a]);
  double* out = s->tmp;
  memset(out, 0, sizeof(double) * s->ncell);
  int di = axis == 0 ? stride : 0, dj = axis == 1 ? stride : 0, dk = axis == 2 ? stride : 0;
  for (int i = lo[0]; i <= hi[0]; i++)
    for (int j = lo[1]; j <= hi[1]; j++)
      for (int k = lo[2]; k <= hi[2]; k++) {
        double l = rd(s, F, i - di, j - dj, k - dk), r = rd(s, F, i + di, j + dj, k + dk);
        out[I3(s, i, j, k)] = alpha * F[I3(s, i, j, k)] + (1.0 - alpha) * 0.5 * (l + r);
      }
  memcpy(F, out, sizeof(double) * s->ncell);
}

/* With a stride set (Sec. 4.1, wide-band filters combining strides): along each axis, for each stride
 * of the set in turn, the n passes and the compensation pass at that stride. */
static void filter_component(o3_sim* s, int comp, double* F) {
  int n = s->c.filter_passes;
  int set[4] = { s->c.filter_stride, 0, 0, 0 };
  if (s->c.filter_strides[0] > 0) for (int q = 0; q < 4; q++) set[q] = s->c.filter_strides[q];
  for (int axis = 0; axis < 3; axis++)
    for (int q = 0; q < 4 && set[q] > 0; q++) {
      for (int p = 0; p < n; p++) filter_pass_axis(s, comp, F, axis, set[q], 0.5);
      if (s->c.filter_compensate) filter_pass_axis(s, comp, F, axis, set[q], 0.5 * n + 1.0);
    }
}

void o3_filter_field(o3_sim* s, int comp, double* F) { filter_component(s, comp, F); }

/* 'Momentum conserving' gather (Sec. 5): the staggered gather copy interpolated to the nodes, the mean of
 * the two nearest values along each half-integer axis of the component (four along two axes); values
 * off the grid count as zero. */
static void to_nodes(o3_sim* s, int comp, double* F) {
  int h[3] = { SX[comp] != 0.0, SY[comp] != 0.0, SZ[comp] != 0.0 };
  double* out = s->tmp;
  for (int i = 0; i <= s->c.nx; i++)
    for (int j = 0; j <= s->c.ny; j++)
      for (int k = 0; k <= s->c.nz; k++) {
        double acc = 0.0;
        int cnt = 0;
        for (int a = 0; a <= h[0]; a++)
          for (int b = 0; b <= h[1]; b++)
            for (int c = 0; c <= h[2]; c++) {
              acc += rd(s, F, i - h[0] + a, j - h[1] + b, k - h[2] + c);
              cnt++;
            }
        out[I3(s, i, j, k)] = acc / cnt;
      }
  memcpy(F, out, sizeof(double) * s->ncell);
}

/* ------------------------------------------------------------------ */
static void gather(const o3_sim* s, double x, double y, double z, double* E, double* B) {
  int ord = s->c.order;
  double X = x / s->dx, Y = y / s->dy, Z = z / s->dz;
  int fx = (int)floor(X), fy = (int)floor(Y), fz = (int)floor(Z);
  const double* src[6] = { s->fE[0], s->fE[1], s->fE[2], s->fB[0], s->fB[1], s->fB[2] };
  double out[6];
  for (int c = 0; c < 6; c++) {
    double acc = 0.0;
    for (int i = fx - 3; i <= fx + 3; i++) {
      const int nod = s->c.gather_nodal;
      double wx = orc_shape(ord, X - (i + (nod ? 0.0 : SX[c])));
      if (wx == 0.0) continue;
      for (int j = fy - 3; j <= fy + 3; j++) {
        double wy = orc_shape(ord, Y - (j + (nod ? 0.0 : SY[c])));
        if (wy == 0.0) continue;
        for (int k = fz - 3; k <= fz + 3; k++) {
          double wz = orc_shape(ord, Z - (k + (nod ? 0.0 : SZ[c])));
          if (wz == 0.0) continue;
          acc += rd(s, src[c], i, j, k) * wx * wy * wz;
        }
      }
    }
    out[c] = acc;
  }
  for (int c = 0; c < 3; c++) { E[c] = out[c]; B[c] = out[3 + c]; }
}

/* ------------------------------------------------------------------ */
/* Esirkepov deposition in 3D (Esirkepov 2001, Sec. 4.2.2) of charge*weight qw moving from p0 to p1:
 * W_x = DS_x (S0_y S0_z + DS_y S0_z/2 + S0_y DS_z/2 + DS_y DS_z/3) and cyclic; J_x(i+1/2) - J_x(i-1/2)
 * = -qw/(dy dz dt) W_x(i), likewise for y and z. */
#define EW 9
static void esirkepov3(o3_sim* s, const double* p0, const double* p1, double qw) {
  int ord = s->c.order;
  double d[3] = { s->dx, s->dy, s->dz };
  int nn[3] = { s->c.nx, s->c.ny, s->c.nz };
  int base[3];
  double S0[3][EW], DS[3][EW];
  for (int a = 0; a < 3; a++) {
    double A0 = p0[a] / d[a], A1 = p1[a] / d[a];
    base[a] = (int)floor(A0 < A1 ? A0 : A1) - 3;
    for (int m = 0; m < EW; m++) {
      S0[a][m] = orc_shape(ord, A0 - (base[a] + m));
      DS[a][m] = orc_shape(ord, A1 - (base[a] + m)) - S0[a][m];
    }
  }
  double* J[3] = { s->F[QJX], s->F[QJY], s->F[QJZ] };
  for (int q = 0; q < 3; q++) {
    int u = (q + 1) % 3, v = (q + 2) % 3;
    double cq = -qw * d[q] / (d[0] * d[1] * d[2] * s->dt);   /* -qw / (d_u d_v dt) */
    for (int mu = 0; mu < EW; mu++)
      for (int mv = 0; mv < EW; mv++) {
        double tr = S0[u][mu] * S0[v][mv] + 0.5 * DS[u][mu] * S0[v][mv] + 0.5 * S0[u][mu] * DS[v][mv]
                    + DS[u][mu] * DS[v][mv] / 3.0;
        double acc = 0.0;
        for (int mq = 0; mq < EW; mq++) {
          acc += cq * DS[q][mq] * tr;
          int idx[3];
          idx[q] = base[q] + mq; idx[u] = base[u] + mu; idx[v] = base[v] + mv;
          if (acc == 0.0) continue;
          if (idx[0] < 0 || idx[0] > nn[0] || idx[1] < 0 || idx[1] > nn[1] || idx[2] < 0 || idx[2] > nn[2]) continue;
          J[q][I3(s, idx[0], idx[1], idx[2])] += acc;
        }
      }
  }
}

/* weights of the test beam (macro-particle counts), in the order it was given */
void o3_beam_weights(o3_sim* s, const double* w) {
  o3_species* b = &s->sp[2];
  for (long j = 0; j < b->n; j++) b->w[j] = w[j];
}

void o3_rho_one(const o3_sim* s, double* rho, double x, double y, double z, double qw);

void o3_deposit_one(o3_sim* s, double x0, double y0, double z0, double x1, double y1, double z1, double qw) {
  double p0[3] = { x0, y0, z0 }, p1[3] = { x1, y1, z1 };
  esirkepov3(s, p0, p1, qw);
}

static void deposit_rho(const o3_sim* s, double* rho, double x, double y, double z, double qw) {
  int ord = s->c.order;
  double X = x / s->dx, Y = y / s->dy, Z = z / s->dz;
  int fx = (int)floor(X), fy = (int)floor(Y), fz = (int)floor(Z);
  for (int i = fx - 3; i <= fx + 3; i++)
    for (int j = fy - 3; j <= fy + 3; j++)
      for (int k = fz - 3; k <= fz + 3; k++) {
        double w = orc_shape(ord, X - i) * orc_shape(ord, Y - j) * orc_shape(ord, Z - k);
        if (w != 0.0 && i >= 0 && i <= s->c.nx && j >= 0 && j <= s->c.ny && k >= 0 && k <= s->c.nz)
          rho[I3(s, i, j, k)] += qw * w / (s->dx * s->dy * s->dz);
      }
}

void o3_rho_one(const o3_sim* s, double* rho, double x, double y, double z, double qw) { deposit_rho(s, rho, x, y, z, qw); }

/* ------------------------------------------------------------------ */
static void sp_reserve(o3_species* p, long n) {
  if (n <= p->cap) return;
  long cap = p->cap ? p->cap : 1024;
  while (cap < n) cap *= 2;
#define RE(f, T) p->f = (T*)realloc(p->f, sizeof(T) * cap)
  RE(x, double); RE(y, double); RE(z, double); RE(ux, double); RE(uy, double); RE(uz, double); RE(w, double);
  RE(id, uint32_t); RE(alive, int);
  RE(tc, double); RE(zf0, double); RE(uxb, double); RE(uyb, double); RE(uzb, double); RE(active, int);
  RE(zl, double);
#undef RE
  p->cap = cap;
}

static void sp_push(o3_species* p, double x, double y, double z, double ux, double uy, double uz, double w, uint32_t id) {
  sp_reserve(p, p->n + 1);
  long j = p->n++;
  p->x[j] = x; p->y[j] = y; p->z[j] = z; p->ux[j] = ux; p->uy[j] = uy; p->uz[j] = uz; p->w[j] = w;
  p->id[j] = id; p->alive[j] = 1;
  p->tc[j] = 0; p->zf0[j] = 0; p->uxb[j] = 0; p->uyb[j] = 0; p->uzb[j] = 0; p->active[j] = 1; p->zl[j] = 0;
}

static void sp_compact(o3_species* p) {
  long o = 0;
  for (long j = 0; j < p->n; j++) {
    if (!p->alive[j]) continue;
    if (o != j) {
      p->x[o] = p->x[j]; p->y[o] = p->y[j]; p->z[o] = p->z[j];
      p->ux[o] = p->ux[j]; p->uy[o] = p->uy[j]; p->uz[o] = p->uz[j];
      p->w[o] = p->w[j]; p->id[o] = p->id[j]; p->alive[o] = 1;
      p->tc[o] = p->tc[j]; p->zf0[o] = p->zf0[j]; p->uxb[o] = p->uxb[j]; p->uyb[o] = p->uyb[j];
      p->uzb[o] = p->uzb[j]; p->active[o] = p->active[j]; p->zl[o] = p->zl[j];
    }
    o++;
  }
  p->n = o;
}

static double time_of(const o3_sim* s, long n) { return (double)n * s->dt; }

o3_sim* o3_create(const o3_config* cfg) {
  o3_sim* s = (o3_sim*)calloc(1, sizeof(o3_sim));
  s->c = *cfg;
  s->gamma = cfg->gamma_boost < 1.0 ? 1.0 : cfg->gamma_boost;
  s->beta = sqrt(1.0 - 1.0 / (s->gamma * s->gamma));
  s->dz = (1.0 + s->beta) * s->gamma * cfg->dz_lab;   /* Sec. 5.1.1 */
  s->dx = cfg->dx; s->dy = cfg->dy;
  if (cfg->dt_override > 0.0) s->dt = cfg->dt_override;
  else s->dt = cfg->courant * orc_cfl_3d(cfg->ck_alpha, cfg->ck_beta, cfg->ck_gamma, s->dx, s->dy, s->dz, cfg->theta);
  s->nxp = cfg->nx + 1; s->nyp = cfg->ny + 1; s->nzp = cfg->nz + 1;
  s->ncell = (long)s->nxp * s->nyp * s->nzp;
#define AL() (double*)calloc(s->ncell, sizeof(double))
  for (int c = 0; c < QNCOMP; c++) s->F[c] = AL();
  for (int c = 0; c < 3; c++) {
    s->Ep[c] = AL(); s->Eb[c] = AL(); s->Ee[c] = AL(); s->Bold[c] = AL(); s->fE[c] = AL(); s->fB[c] = AL();
    s->Es[c][0] = AL(); s->Es[c][1] = AL(); s->Bs[c][0] = AL(); s->Bs[c][1] = AL();
  }
  s->tmp = AL();
#undef AL
  int nn[3] = { cfg->nx, cfg->ny, cfg->nz };
  int per[3] = { cfg->periodic_x, cfg->periodic_y, cfg->periodic_z };
  double dd[3] = { s->dx, s->dy, s->dz };
  for (int a = 0; a < 3; a++) {
    s->s_int[a] = (double*)calloc(nn[a] + 2, sizeof(double));
    s->s_half[a] = (double*)calloc(nn[a] + 2, sizeof(double));
    for (int i = 0; i <= nn[a]; i++) {
      s->s_int[a][i] = per[a] ? 0.0 : pml_sigma(s, i, nn[a], dd[a]);
      s->s_half[a][i] = per[a] ? 0.0 : pml_sigma(s, i + 0.5, nn[a], dd[a]);
    }
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
  for (int a = 0; a < 3; a++) { s->glo[a] = L + g; s->ghi[a] = nn[a] - L - g; }
  s->sp[0].q = -O_QE; s->sp[0].m = O_ME;
  s->sp[1].q = O_QE;  s->sp[1].m = 1836.15267343 * O_ME;
  s->sp[2].q = -O_QE; s->sp[2].m = O_ME;
  return s;
}

void o3_destroy(o3_sim* s) {
  if (!s) return;
  for (int c = 0; c < QNCOMP; c++) free(s->F[c]);
  for (int c = 0; c < 3; c++) {
    free(s->Ep[c]); free(s->Eb[c]); free(s->Ee[c]); free(s->Bold[c]); free(s->fE[c]); free(s->fB[c]);
    free(s->Es[c][0]); free(s->Es[c][1]); free(s->Bs[c][0]); free(s->Bs[c][1]);
  }
  free(s->tmp);
  for (int a = 0; a < 3; a++) { free(s->s_int[a]); free(s->s_half[a]); }
  for (int j = 0; j < 3; j++) {
    o3_species* p = &s->sp[j];
    free(p->x); free(p->y); free(p->z); free(p->ux); free(p->uy); free(p->uz); free(p->w); free(p->id);
    free(p->alive); free(p->tc); free(p->zf0); free(p->uxb); free(p->uyb); free(p->uzb); free(p->active); free(p->zl);
  }
  free(s->delta);
  free(s->rzL); free(s->rtL); free(s->rout); free(s->rdone);
  free(s);
}

/* info: dx, dy, dz, dt, gamma, beta, step, t, guard, then (lo, hi) of the particle domain per axis */
void o3_info(const o3_sim* s, double* out) {
  out[0] = s->dx; out[1] = s->dy; out[2] = s->dz; out[3] = s->dt; out[4] = s->gamma; out[5] = s->beta;
  out[6] = (double)s->step; out[7] = time_of(s, s->step); out[8] = s->c.particle_guard;
  for (int a = 0; a < 3; a++) { out[9 + 2 * a] = s->glo[a]; out[10 + 2 * a] = s->ghi[a]; }
  out[15] = s->beam_vbar;
}

/* ------------------------------------------------------------------ */
/* Plasma (Sec. 3.1.1, PR-9, PR-12) on a lattice of ppc_x x ppc_y x ppc_z per cell: row m at
 * z'_m(t) = (m + 1/2) h - beta c t, h = dz/ppc_z, density gamma n0(gamma (m + 1/2) h); weight
 * w = n' dx dy dz/(ppc_x ppc_y ppc_z); id = m (nxl nyl) + a nyl + b (32-bit). */
static double lab_density(const o3_plasma* p, double zl) {
  if (zl < p->z_start_lab) return 0.0;
  double r = zl - p->z_start_lab;
  if (p->ramp_lab > 0.0 && r < p->ramp_lab) return p->n0 * r / p->ramp_lab;
  double plateau_end = p->ramp_lab + p->length_lab;
  if (p->length_lab > 0.0 && r >= plateau_end) return 0.0;
  return p->n0;
}

static double z_hi_of(const o3_sim* s) { return s->ghi[2] * s->dz; }
static double z_lo_of(const o3_sim* s) { return s->glo[2] * s->dz; }

static long rows_inside(const o3_sim* s, double t) {
  return (long)ceil((z_hi_of(s) + s->beta * O_C * t) / s->h_row - 0.5);
}

static void add_row(o3_sim* s, long m, double t) {
  double zlat = (m + 0.5) * s->h_row;
  double n = s->gamma * lab_density(&s->pl, s->gamma * zlat);
  if (n <= 0.0) return;
  double zp = zlat - s->beta * O_C * t;
  double w = n * s->dx * s->dy * s->dz / (double)(s->pl.ppc_x * s->pl.ppc_y * s->pl.ppc_z);
  double uz = -s->gamma * s->beta * O_C;
  for (long a = 0; a < s->nxl; a++)
    for (long b = 0; b < s->nyl; b++) {
      double xp = (s->glo[0] + (a + 0.5) / s->pl.ppc_x) * s->dx;
      double yp = (s->glo[1] + (b + 0.5) / s->pl.ppc_y) * s->dy;
      uint32_t id = (uint32_t)((uint64_t)m * (uint64_t)(s->nxl * s->nyl) + (uint64_t)(a * s->nyl + b));
      sp_push(&s->sp[0], xp, yp, zp, 0.0, 0.0, uz, w, id);
      if (s->pl.ions) {
        sp_push(&s->sp[1], xp, yp, zp, 0.0, 0.0, uz, w, id);
        s->sp[1].zl[s->sp[1].n - 1] = zlat;
      }
    }
}

int o3_load_plasma(o3_sim* s, const o3_plasma* p) {
  s->pl = *p; s->has_plasma = 1;
  s->h_row = s->dz / p->ppc_z;
  s->nxl = (long)(s->ghi[0] - s->glo[0]) * p->ppc_x;
  s->nyl = (long)(s->ghi[1] - s->glo[1]) * p->ppc_y;
  double t = time_of(s, s->step);
  long m_end = rows_inside(s, t);
  long m_beg = (long)ceil((z_lo_of(s) + s->beta * O_C * t) / s->h_row - 0.5);
  for (long m = m_beg; m < m_end; m++) add_row(s, m, t);
  s->row_next = m_end;
  return 0;
}

/* ------------------------------------------------------------------ */
/* Laser (Sec. 3.1.2): the antenna at rest in the computational frame emits the lab waveform
 * E0 exp(-((x-xc)^2+(y-yc)^2)/w0^2) exp(-(s-t_peak)^2/(2 sigma_t^2)) sin(omega (s - t_peak) + phase),
 * Doppler-scaled, E_emit = g(x, y, t'/((1+beta) gamma))/((1+beta) gamma) (PR-14), as a surface
 * current K_y = -2 eps0 c E_emit (PR-13). One pair of opposite macro-particles per transverse node
 * (i, j) of the particle domain: the negative partner stays at (x_i, y_j, z_a); the positive one, of
 * charge Q = 200 eps0 E0 dx dy/((1+beta) gamma) (so that its speed stays below c/100), moves along y
 * with v = K dx dy/Q and deposits with Esirkepov; the pair's charge is in Gauss's law. */
int o3_set_laser(o3_sim* s, const o3_laser* l) {
  s->las = *l; s->has_laser = 1;
  double om = 2.0 * O_PI * O_C / l->lambda0;
  double E0 = l->a0 * O_ME * O_C * om / O_QE;
  double dop = (1.0 + s->beta) * s->gamma;
  s->q_pair = 200.0 * O_EPS0 * E0 * s->dx * s->dy / dop;
  free(s->delta);
  s->delta = (double*)calloc((size_t)s->nxp * s->nyp, sizeof(double));
  return 0;
}

static double emit_field(const o3_sim* s, double x, double y, double tp) {
  const o3_laser* l = &s->las;
  double om = 2.0 * O_PI * O_C / l->lambda0;
  double E0 = l->a0 * O_ME * O_C * om / O_QE;
  double dop = (1.0 + s->beta) * s->gamma;
  double sl = tp / dop;
  double sig = l->tau_fwhm / (2.0 * sqrt(log(2.0)));
  double dx = x - l->x_center, dy = y - l->y_center;
  double g = E0 * exp(-(dx * dx + dy * dy) / (l->w0 * l->w0)) *
             exp(-(sl - l->t_peak) * (sl - l->t_peak) / (2.0 * sig * sig)) * sin(om * (sl - l->t_peak) + l->phase);
  return g / dop;
}

static int antenna_inside(const o3_sim* s) {
  double za = s->las.z_antenna;
  return za >= z_lo_of(s) && za < z_hi_of(s);
}

static void antenna(o3_sim* s) {
  if (!s->has_laser || !antenna_inside(s)) return;
  double th = time_of(s, s->step) + 0.5 * s->dt;
  for (int i = s->glo[0]; i <= s->ghi[0]; i++)
    for (int j = s->glo[1]; j <= s->ghi[1]; j++) {
      double K = -2.0 * O_EPS0 * O_C * emit_field(s, i * s->dx, j * s->dy, th);
      double v = K * s->dx * s->dy / s->q_pair;
      double* dl = &s->delta[(long)i * s->nyp + j];
      double p0[3] = { i * s->dx, j * s->dy + *dl, s->las.z_antenna };
      double p1[3] = { i * s->dx, j * s->dy + *dl + v * s->dt, s->las.z_antenna };
      if (v != 0.0) esirkepov3(s, p0, p1, s->q_pair);
      *dl += v * s->dt;
    }
}

/* ------------------------------------------------------------------ */
/* Test beam through a plane (Sec. 3.1.1), as in 2D with the y coordinate carried along. */
int o3_set_beam(o3_sim* s, long n, const double* x, const double* y, const double* z, const double* ux,
                const double* uy, const double* uz, double t_lab, double z_plane) {
  o3_species* b = &s->sp[2];
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
    double tcross = t_lab + (z_plane - z[j]) / vz;
    double xs = x[j] + vx * (tcross - t_lab), ys = y[j] + vy * (tcross - t_lab);
    double tpc = g * (tcross - be * z_plane / O_C);
    double zpc = g * (z_plane - be * O_C * tcross);
    double den = 1.0 - be * betab;
    double vxp = vx / (g * den), vyp = vy / (g * den), vzp = (vz - be * O_C) / den;
    vpsum += vzp;
    double v2 = (vxp * vxp + vyp * vyp + vzp * vzp) / (O_C * O_C);
    double gp = 1.0 / sqrt(1.0 - v2);
    sp_push(b, xs, ys, 0.0, gp * vxp, gp * vyp, gp * vzp, 1.0, (uint32_t)j);
    tcv[j] = tpc; zcv[j] = zpc;
  }
  double vbar = vpsum / n;
  for (long j = 0; j < n; j++) {
    long q = b->n - n + j;
    b->tc[q] = tcv[j];
    b->zf0[q] = zcv[j] - vbar * tcv[j];
    b->uxb[q] = b->ux[q]; b->uyb[q] = b->uy[q]; b->uzb[q] = b->uz[q];
    b->active[q] = 0;
    b->z[q] = b->zf0[q] + vbar * time_of(s, s->step);
  }
  free(tcv); free(zcv);
  s->beam_vbar = vbar; s->has_beam = 1;
  return 0;
}

/* ------------------------------------------------------------------ */
/* lab-frame sample rows (Sec. 3.2, PR-16), each a transverse slice of 6 x (nx+1) x (ny+1) values */
int o3_btd_set(o3_sim* s, int nrows, const double* zL, const double* tL) {
  free(s->rzL); free(s->rtL); free(s->rout); free(s->rdone);
  s->nrows = nrows;
  s->rzL = (double*)malloc(sizeof(double) * nrows); s->rtL = (double*)malloc(sizeof(double) * nrows);
  memcpy(s->rzL, zL, sizeof(double) * nrows); memcpy(s->rtL, tL, sizeof(double) * nrows);
  s->rout = (double*)calloc((size_t)nrows * 6 * s->nxp * s->nyp, sizeof(double));
  s->rdone = (int*)calloc((size_t)nrows * 2, sizeof(int));
  return 0;
}

static double interp_z(const o3_sim* s, const double* F, int i, int j, double zp, double stz) {
  double Z = zp / s->dz - stz;
  int k = (int)floor(Z);
  double f = Z - k;
  return (1.0 - f) * rd(s, F, i, j, k) + f * rd(s, F, i, j, k + 1);
}

static void btd_accumulate(o3_sim* s, int which, int post) {
  double g = s->gamma, be = s->beta;
  long plane = (long)s->nxp * s->nyp;
  for (int r = 0; r < s->nrows; r++) {
    double tp = g * (s->rtL[r] - be * s->rzL[r] / O_C);
    double zp = g * (s->rzL[r] - be * O_C * s->rtL[r]);
    double ta, tb;
    if (which == 0) { ta = time_of(s, s->step); tb = time_of(s, s->step + 1); }
    else { ta = time_of(s, s->step) - 0.5 * s->dt; tb = ta + s->dt; }
    if (!(tp >= ta && tp < tb)) continue;
    double f = (tp - ta) / s->dt;
    double wgt = post ? f : 1.0 - f;
    double* out = s->rout + (size_t)r * 6 * plane;
    for (int i = 0; i <= s->c.nx; i++)
      for (int j = 0; j <= s->c.ny; j++) {
        long o = (long)i * s->nyp + j;
        if (which == 0) {
          double ex = interp_z(s, s->F[QEX], i, j, zp, SZ[QEX]);
          double ey = interp_z(s, s->F[QEY], i, j, zp, SZ[QEY]);
          double ez = interp_z(s, s->F[QEZ], i, j, zp, SZ[QEZ]);
          out[0 * plane + o] += wgt * g * ex;
          out[1 * plane + o] += wgt * g * ey;
          out[2 * plane + o] += wgt * ez;
          out[3 * plane + o] += wgt * (-g * be * ey / O_C);
          out[4 * plane + o] += wgt * (g * be * ex / O_C);
        } else {
          double bx = interp_z(s, s->F[QBX], i, j, zp, SZ[QBX]);
          double by = interp_z(s, s->F[QBY], i, j, zp, SZ[QBY]);
          double bz = interp_z(s, s->F[QBZ], i, j, zp, SZ[QBZ]);
          out[0 * plane + o] += wgt * g * be * O_C * by;
          out[1 * plane + o] += wgt * (-g * be * O_C * bx);
          out[3 * plane + o] += wgt * g * bx;
          out[4 * plane + o] += wgt * g * by;
          out[5 * plane + o] += wgt * bz;
        }
      }
    if (post) s->rdone[2 * r + which] = 1;
  }
}

int o3_btd_get(const o3_sim* s, double* out, int* done) {
  memcpy(out, s->rout, sizeof(double) * (size_t)s->nrows * 6 * s->nxp * s->nyp);
  memcpy(done, s->rdone, sizeof(int) * (size_t)s->nrows * 2);
  return 0;
}

/* ------------------------------------------------------------------ */
/* One PIC step in the order of PR-1. */
static void one_step(o3_sim* s) {
  btd_accumulate(s, 0, 0);
  btd_accumulate(s, 1, 0);
  faraday(s);
  for (int c = 0; c < 3; c++)
    for (long p = 0; p < s->ncell; p++) {
      s->fE[c][p] = s->F[QEX + c][p];
      s->fB[c][p] = 0.5 * (s->Bold[c][p] + s->F[QBX + c][p]);
    }
  if (s->c.filter_gather)
    for (int c = 0; c < 3; c++) { filter_component(s, QEX + c, s->fE[c]); filter_component(s, QBX + c, s->fB[c]); }
  if (s->c.gather_nodal)
    for (int c = 0; c < 3; c++) { to_nodes(s, QEX + c, s->fE[c]); to_nodes(s, QBX + c, s->fB[c]); }
  for (int c = QJX; c <= QJZ; c++) memset(s->F[c], 0, sizeof(double) * s->ncell);
  double lo[3], hi[3];
  double dd[3] = { s->dx, s->dy, s->dz };
  for (int a = 0; a < 3; a++) { lo[a] = s->glo[a] * dd[a]; hi[a] = s->ghi[a] * dd[a]; }
  hi[2] += s->dz;
  double tn = time_of(s, s->step), tn1 = time_of(s, s->step + 1);
  for (int sp = 0; sp < 3; sp++) {
    o3_species* p = &s->sp[sp];
    for (long q = 0; q < p->n; q++) {
      if (!p->alive[q]) continue;
      if (sp == 2 && !p->active[q]) {
        if (tn >= p->tc[q]) {
          p->active[q] = 1;
          p->ux[q] = p->uxb[q]; p->uy[q] = p->uyb[q]; p->uz[q] = p->uzb[q];
          if (p->x[q] < lo[0] || p->x[q] >= hi[0] || p->y[q] < lo[1] || p->y[q] >= hi[1] ||
              p->z[q] < lo[2] || p->z[q] >= hi[2]) { p->alive[q] = 0; continue; }
        } else {
          const double zn = p->zf0[q] + s->beam_vbar * tn1;
          /* a frozen particle inside the particle domain carries its charge along z at the mean velocity */
          if (s->c.beam_self && p->x[q] >= lo[0] && p->x[q] < hi[0] && p->y[q] >= lo[1] && p->y[q] < hi[1] &&
              p->z[q] >= lo[2] && p->z[q] < hi[2] && zn >= lo[2] && zn < hi[2]) {
            double p0[3] = { p->x[q], p->y[q], p->z[q] }, p1[3] = { p->x[q], p->y[q], zn };
            esirkepov3(s, p0, p1, p->q * p->w[q]);
          }
          p->z[q] = zn;
          continue;
        }
      }
      double u[3] = { p->ux[q], p->uy[q], p->uz[q] };
      if (sp != 1) {
        double E[3], B[3];
        gather(s, p->x[q], p->y[q], p->z[q], E, B);
        orc_boris(u, E, B, p->q, p->m, s->dt);
      }
      double gm = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (O_C * O_C));
      double pn[3] = { p->x[q] + s->dt * u[0] / gm, p->y[q] + s->dt * u[1] / gm, p->z[q] + s->dt * u[2] / gm };
      if (sp == 1) {   /* ions fixed in the lab (PR-9, PR-12) */
        pn[0] = p->x[q]; pn[1] = p->y[q];
        p->z[q] = p->zl[q] - s->beta * O_C * tn;
        pn[2] = p->zl[q] - s->beta * O_C * tn1;
      }
      if (sp != 2 || s->c.beam_self) {
        double p0[3] = { p->x[q], p->y[q], p->z[q] };
        esirkepov3(s, p0, pn, p->q * p->w[q]);
      }
      p->x[q] = pn[0]; p->y[q] = pn[1]; p->z[q] = pn[2];
      p->ux[q] = u[0]; p->uy[q] = u[1]; p->uz[q] = u[2];
      if (pn[0] < lo[0] || pn[0] >= hi[0] || pn[1] < lo[1] || pn[1] >= hi[1] || pn[2] < lo[2] || pn[2] >= hi[2])
        p->alive[q] = 0;
    }
  }
  antenna(s);
  if (s->c.filter_J) for (int c = 0; c < 3; c++) filter_component(s, QJX + c, s->F[QJX + c]);
  ampere(s);
  btd_accumulate(s, 0, 1);
  btd_accumulate(s, 1, 1);
  sp_compact(&s->sp[0]); sp_compact(&s->sp[1]);
  if (s->has_plasma) {
    long m_end = rows_inside(s, tn1);
    for (long m = s->row_next; m < m_end; m++) add_row(s, m, tn1);
    if (m_end > s->row_next) s->row_next = m_end;
  }
  s->step++;
}

int o3_step(o3_sim* s, int n) {
  for (int i = 0; i < n; i++) one_step(s);
  return 0;
}

/* ------------------------------------------------------------------ */
void o3_get_field(const o3_sim* s, int comp, double* out) { memcpy(out, s->F[comp], sizeof(double) * s->ncell); }
void o3_set_field(o3_sim* s, int comp, const double* in) { memcpy(s->F[comp], in, sizeof(double) * s->ncell); }
void o3_get_gather_field(const o3_sim* s, int comp, double* out) {
  memcpy(out, comp < 3 ? s->fE[comp] : s->fB[comp - 3], sizeof(double) * s->ncell);
}
long o3_num_particles(const o3_sim* s, int species) { return s->sp[species].n; }
void o3_get_particles(const o3_sim* s, int species, double* x, double* y, double* z, double* ux, double* uy,
                      double* uz, double* w, uint32_t* id, int* flag) {
  const o3_species* p = &s->sp[species];
  for (long j = 0; j < p->n; j++) {
    x[j] = p->x[j]; y[j] = p->y[j]; z[j] = p->z[j]; ux[j] = p->ux[j]; uy[j] = p->uy[j]; uz[j] = p->uz[j];
    w[j] = p->w[j]; id[j] = p->id[j]; flag[j] = (p->alive[j] ? 1 : 0) | (p->active[j] ? 2 : 0);
  }
}
void o3_set_particles(o3_sim* s, int species, long n, const double* x, const double* y, const double* z,
                      const double* ux, const double* uy, const double* uz, const double* w) {
  o3_species* p = &s->sp[species];
  p->n = 0;
  for (long j = 0; j < n; j++) sp_push(p, x[j], y[j], z[j], ux[j], uy[j], uz[j], w[j], (uint32_t)j);
}

/* charge density of the plasma species and of the antenna pairs */
void o3_rho(const o3_sim* s, double* rho) {
  memset(rho, 0, sizeof(double) * s->ncell);
  for (int j = 0; j < 2; j++) {
    const o3_species* p = &s->sp[j];
    for (long q = 0; q < p->n; q++)
      if (p->alive[q]) deposit_rho(s, rho, p->x[q], p->y[q], p->z[q], p->q * p->w[q]);
  }
  if (s->has_laser && antenna_inside(s))
    for (int i = s->glo[0]; i <= s->ghi[0]; i++)
      for (int j = s->glo[1]; j <= s->ghi[1]; j++) {
        double dl = s->delta[(long)i * s->nyp + j];
        if (dl == 0.0) continue;
        deposit_rho(s, rho, i * s->dx, j * s->dy + dl, s->las.z_antenna, s->q_pair);
        deposit_rho(s, rho, i * s->dx, j * s->dy, s->las.z_antenna, -s->q_pair);
      }
}

/* out = [n_e, n_beam_active, <gamma_lab>, rms/mean, field energy [J]] */
void o3_diag(const o3_sim* s, double* out) {
  const o3_species* b = &s->sp[2];
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
    double e2 = s->F[QEX][p] * s->F[QEX][p] + s->F[QEY][p] * s->F[QEY][p] + s->F[QEZ][p] * s->F[QEZ][p];
    double b2 = s->F[QBX][p] * s->F[QBX][p] + s->F[QBY][p] * s->F[QBY][p] + s->F[QBZ][p] * s->F[QBZ][p];
    en += 0.5 * (O_EPS0 * e2 + b2 / O_MU0) * s->dx * s->dy * s->dz;
  }
  out[0] = (double)s->sp[0].n; out[1] = (double)na; out[2] = mean;
  out[3] = mean > 0 ? sqrt(var > 0 ? var : 0) / mean : 0.0; out[4] = en;
}
