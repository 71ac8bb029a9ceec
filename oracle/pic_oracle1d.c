/*
 * FP64 CPU oracle of the boosted-frame electromagnetic PIC step in one dimension (z; fields and particle
 * positions depend on z only, the three momentum components are kept).
 *
 * TEST INFRASTRUCTURE ONLY. Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference arm of bench.py may load this library. The product
 * path (the CUDA library behind include/pic.h) neither links nor calls it, and
 * this file includes no header of the product.
 *
 * The method of the paper (Vay et al., arXiv:1009.2727) in 1D, as App. I writes it (Eq. 1db-1de) for
 * the transverse pair and as the 3D scheme gives it for every component with d/dx = d/dy = 0:
 *   - Faraday:  dBx/dt = +dEy/dz, dBy/dt = -dEx/dz, Bz constant (the enlarged operator reduces to
 *               the Yee difference: alpha + 4 beta + 4 gamma = 1), with Friedman's E_eff (Sec. 4.3);
 *   - Ampere:   dEx/dt = -c^2 dBy/dz - Jx/eps0, dEy/dt = c^2 dBx/dz - Jy/eps0, dEz/dt = -Jz/eps0;
 *   - PML (App. II) at both ends along z (in 1D each component has a single part);
 *   - filter (Sec. 4.1) along z: passes, compensation, stride or a set of strides;
 *   - Esirkepov deposition in 1D: Jz from the charge flux, Jx and Jy from the velocity times the mean of
 *     the old and new shapes (Esirkepov 2001, Sec. 4.2.2);
 *   - cubic (or linear) B-splines, the gather from the Yee locations or from node-interpolated fields
 *     (Sec. 5); Boris push (orc_boris of pic_oracle.c, same library);
 *   - plasma rows through the plane z_hi, ions fixed in the lab, a current-sheet antenna (Sec. 3.1),
 *     a moving window in the lab frame (App. I's scaled stage).
 *
 * Layout: node k of every nz+1 array at index k. Yee positions along z: Ex, Ey, Bz, Jx, Jy at k;
 * Ez, Bx, By, Jz at k + 1/2. Weights are per unit transverse area.
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
void orc_boris(double* u, const double* E, const double* B, double q, double m, double dt);

enum { WEX = 0, WEY, WEZ, WBX, WBY, WBZ, WJX, WJY, WJZ, WNCOMP };

typedef struct {
  int nz;
  double dz_lab, gamma_boost, courant, dt_override, theta;
  int pml_cells;
  double pml_sigma_max, pml_delta, pml_power;
  int pml_xi_exp;
  int filter_passes, filter_stride, filter_compensate, filter_J, filter_gather;
  int order, particle_guard;
  int moving_window;
  double window_beta;
  int filter_strides[4];
  int gather_nodal;
} o1_config;

typedef struct {
  double n0, z_start_lab, ramp_lab, length_lab;
  int ppc_z, ions;
} o1_plasma;

typedef struct {
  double lambda0, a0, tau_fwhm, t_peak, phase, z_antenna;
} o1_laser;

typedef struct {
  double *z, *ux, *uy, *uz, *w, *zl;
  uint32_t* id;
  int* alive;
  long n, cap;
  double q, m;
} o1_species;

typedef struct {
  o1_config c;
  double dz, dt, gamma, beta, z0;
  long shifts, step;
  int n1;
  double* F[WNCOMP];
  double *Ep[3], *Eb[3], *Ee[3], *Bold[3], *fE[3], *fB[3], *tmp;
  double *s_int, *s_half;
  int glo, ghi;
  o1_species sp[2];      /* 0 electrons, 1 ions */
  o1_plasma pl; int has_plasma;
  long row_next;
  double h_row;
  o1_laser las; int has_laser;
} o1_sim;

/* stagger (cells) of each component along z */
static const double SZ1[WNCOMP] = { 0.0, 0.0, 0.5, 0.5, 0.5, 0.0, 0.0, 0.0, 0.5 };

static double rd(const o1_sim* s, const double* F, int k) {
  if (k < 0 || k > s->c.nz) return 0.0;
  return F[k];
}

/* valid range: a half-staggered index runs 0..nz-1; an integer one 1..nz-1 for E (PEC walls), 0..nz
 * for B */
static void vrange(const o1_sim* s, int comp, int* lo, int* hi) {
  int c = comp >= WJX ? comp - WJX : comp;
  if (SZ1[c] > 0.0) { *lo = 0; *hi = s->c.nz - 1; }
  else if (c < 3) { *lo = 1; *hi = s->c.nz - 1; }
  else { *lo = 0; *hi = s->c.nz; }
}

static double pml_sigma(const o1_sim* s, double pos) {
  int L = s->c.pml_cells, n = s->c.nz;
  if (L <= 0) return 0.0;
  double d = 0.0;
  if (pos < L) d = L - pos;
  if (pos > n - L) d = pos - (n - L);
  if (d <= 0.0) return 0.0;
  return s->c.pml_sigma_max * O_C / s->dz * pow(d / s->c.pml_delta, s->c.pml_power);
}
static double pml_xi(const o1_sim* s, double sig) {
  if (s->c.pml_xi_exp) return exp(-sig * s->dt);
  return (1.0 - 0.5 * sig * s->dt) / (1.0 + 0.5 * sig * s->dt);
}
static double pml_coef(const o1_sim* s, double sig) {
  if (sig <= 0.0) return s->dt;
  return (1.0 - pml_xi(s, sig)) / sig;
}

/* ------------------------------------------------------------------ */
/* Faraday with E_eff (PR-1) and the PML: Bx(k+1/2) += dEy/dz, By(k+1/2) -= dEx/dz over dt. */
static void faraday(o1_sim* s) {
  double th = s->c.theta;
  int n1 = s->n1;
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < n1; k++)
      s->Ee[c][k] = (1.0 + th / 4.0) * s->F[WEX + c][k] - 0.5 * s->Ep[c][k] + (0.5 - th / 4.0) * s->Eb[c][k];
  for (int c = 0; c < 3; c++) memcpy(s->Bold[c], s->F[WBX + c], sizeof(double) * n1);
  for (int q = 0; q < 2; q++) {        /* Bx (q = 0) from Ey, By (q = 1) from Ex */
    int comp = WBX + q, lo, hi;
    vrange(s, comp, &lo, &hi);
    const double* E = s->Ee[q == 0 ? 1 : 0];
    double sgn = q == 0 ? 1.0 : -1.0;
    double* B = s->F[comp];
    for (int k = lo; k <= hi; k++) {
      double d = sgn * (rd(s, E, k + 1) - rd(s, E, k)) / s->dz;
      double sg = s->s_half[k];
      if (sg > 0.0) B[k] = pml_xi(s, sg) * B[k] + pml_coef(s, sg) * d;
      else B[k] = B[k] + s->dt * d;
    }
  }
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < n1; k++) {
      s->Eb[c][k] = (1.0 - th / 2.0) * s->F[WEX + c][k] + (th / 2.0) * s->Eb[c][k];
      s->Ep[c][k] = s->F[WEX + c][k];
    }
}

/* Ampere: Ex(k) += -c^2 dBy/dz - Jx/eps0, Ey(k) += c^2 dBx/dz - Jy/eps0, Ez(k+1/2) += -Jz/eps0 (times
 * dt); in the PML the current is absent and the curl term is damped. */
static void ampere(o1_sim* s) {
  const double c2 = O_C * O_C;
  for (int q = 0; q < 3; q++) {
    int comp = WEX + q, lo, hi;
    vrange(s, comp, &lo, &hi);
    double* E = s->F[comp];
    const double* J = s->F[WJX + q];
    for (int k = lo; k <= hi; k++) {
      double d = 0.0;
      if (q == 0) d = -c2 * (rd(s, s->F[WBY], k) - rd(s, s->F[WBY], k - 1)) / s->dz;
      if (q == 1) d = c2 * (rd(s, s->F[WBX], k) - rd(s, s->F[WBX], k - 1)) / s->dz;
      double sg = q == 2 ? s->s_half[k] : s->s_int[k];
      if (sg > 0.0) E[k] = pml_xi(s, sg) * E[k] + pml_coef(s, sg) * d;
      else E[k] = E[k] + s->dt * (d - J[k] / O_EPS0);
    }
  }
}

/* ------------------------------------------------------------------ */
/* Filter (Sec. 4.1) along z, pass by pass, zero outside the component's valid range */
static void filter_pass(o1_sim* s, int comp, double* F, int stride, double alpha) {
  int lo, hi;
  vrange(s, comp, &lo, &hi);
  double* out = s->tmp;
  memset(out, 0, sizeof(double) * s->n1);
  for (int k = lo; k <= hi; k++)
    out[k] = alpha * F[k] + (1.0 - alpha) * 0.5 * (rd(s, F, k - stride) + rd(s, F, k + stride));
  memcpy(F, out, sizeof(double) * s->n1);
}

static void filter_component(o1_sim* s, int comp, double* F) {
  int n = s->c.filter_passes;
  int set[4] = { s->c.filter_stride, 0, 0, 0 };
  if (s->c.filter_strides[0] > 0) for (int q = 0; q < 4; q++) set[q] = s->c.filter_strides[q];
  for (int q = 0; q < 4 && set[q] > 0; q++) {
    for (int p = 0; p < n; p++) filter_pass(s, comp, F, set[q], 0.5);
    if (s->c.filter_compensate) filter_pass(s, comp, F, set[q], 0.5 * n + 1.0);
  }
}

void o1_filter_field(o1_sim* s, int comp, double* F) { filter_component(s, comp, F); }

/* 'momentum conserving' gather (Sec. 5): a half-staggered copy becomes the mean of its two nearest
 * values at each node */
static void to_nodes(o1_sim* s, int comp, double* F) {
  if (SZ1[comp] == 0.0) return;
  double* out = s->tmp;
  for (int k = 0; k <= s->c.nz; k++) out[k] = 0.5 * (rd(s, F, k - 1) + rd(s, F, k));
  memcpy(F, out, sizeof(double) * s->n1);
}

/* ------------------------------------------------------------------ */
/* field of component c at the particle's position Z (cells from the grid origin) */
static double gather1(const o1_sim* s, const double* F, int c, double Z) {
  double st = s->c.gather_nodal ? 0.0 : SZ1[c];
  int f = (int)floor(Z);
  double acc = 0.0;
  for (int k = f - 3; k <= f + 3; k++) {
    double wz = orc_shape(s->c.order, Z - (k + st));
    if (wz != 0.0) acc += rd(s, F, k) * wz;
  }
  return acc;
}

/* Esirkepov in 1D for charge*weight qw (per unit area) moving Z0 -> Z1 (cells) in dt with transverse
 * velocities vx, vy: Jz(k+1/2) - Jz(k-1/2) = -qw (S1(k) - S0(k)) / dt, Jz zero below the stencil;
 * Jx(k), Jy(k) = qw v (S0(k) + S1(k)) / (2 dz). */
static void esirkepov1(o1_sim* s, double Z0, double Z1, double vx, double vy, double qw) {
  int ord = s->c.order;
  int b = (int)floor(Z0 < Z1 ? Z0 : Z1) - 3;
  double run = 0.0;
  for (int a = 0; a < 9; a++) {
    int k = b + a;
    double S0 = orc_shape(ord, Z0 - k), S1 = orc_shape(ord, Z1 - k);
    run += S1 - S0;
    if (k < 0 || k > s->c.nz) continue;
    s->F[WJZ][k] += -qw * run / s->dt;
    s->F[WJX][k] += qw * vx * 0.5 * (S0 + S1) / s->dz;
    s->F[WJY][k] += qw * vy * 0.5 * (S0 + S1) / s->dz;
  }
}

void o1_deposit_one(o1_sim* s, double z0, double z1, double vx, double vy, double qw) {
  esirkepov1(s, (z0 - s->z0) / s->dz, (z1 - s->z0) / s->dz, vx, vy, qw);
}

/* ------------------------------------------------------------------ */
static void sp_reserve(o1_species* p, long n) {
  if (n <= p->cap) return;
  long c = p->cap ? p->cap : 1024;
  while (c < n) c *= 2;
  p->z = realloc(p->z, c * sizeof(double)); p->zl = realloc(p->zl, c * sizeof(double));
  p->ux = realloc(p->ux, c * sizeof(double)); p->uy = realloc(p->uy, c * sizeof(double));
  p->uz = realloc(p->uz, c * sizeof(double)); p->w = realloc(p->w, c * sizeof(double));
  p->id = realloc(p->id, c * sizeof(uint32_t)); p->alive = realloc(p->alive, c * sizeof(int));
  p->cap = c;
}

static void sp_push(o1_species* p, double z, double ux, double uy, double uz, double w, uint32_t id, double zl) {
  sp_reserve(p, p->n + 1);
  long j = p->n++;
  p->z[j] = z; p->ux[j] = ux; p->uy[j] = uy; p->uz[j] = uz; p->w[j] = w; p->id[j] = id; p->zl[j] = zl;
  p->alive[j] = 1;
}

static void sp_compact(o1_species* p) {
  long o = 0;
  for (long j = 0; j < p->n; j++) {
    if (!p->alive[j]) continue;
    p->z[o] = p->z[j]; p->ux[o] = p->ux[j]; p->uy[o] = p->uy[j]; p->uz[o] = p->uz[j];
    p->w[o] = p->w[j]; p->id[o] = p->id[j]; p->zl[o] = p->zl[j]; p->alive[o] = 1;
    o++;
  }
  p->n = o;
}

static double time_of(const o1_sim* s, long n) { return (double)n * s->dt; }

/* CFL limit in 1D: c dt <= dz, times sqrt((2 + theta)/(2 + 3 theta)) with Friedman damping */
o1_sim* o1_create(const o1_config* cfg) {
  o1_sim* s = calloc(1, sizeof(o1_sim));
  s->c = *cfg;
  s->gamma = cfg->gamma_boost < 1.0 ? 1.0 : cfg->gamma_boost;
  s->beta = sqrt(1.0 - 1.0 / (s->gamma * s->gamma));
  s->dz = (1.0 + s->beta) * s->gamma * cfg->dz_lab;      /* Sec. 5.1.1 */
  double th = cfg->theta;
  double lim = s->dz / O_C * sqrt((2.0 + th) / (2.0 + 3.0 * th));
  s->dt = cfg->dt_override > 0.0 ? cfg->dt_override : cfg->courant * lim;
  s->n1 = cfg->nz + 1;
  for (int c = 0; c < WNCOMP; c++) s->F[c] = calloc(s->n1, sizeof(double));
  for (int c = 0; c < 3; c++) {
    s->Ep[c] = calloc(s->n1, sizeof(double)); s->Eb[c] = calloc(s->n1, sizeof(double));
    s->Ee[c] = calloc(s->n1, sizeof(double)); s->Bold[c] = calloc(s->n1, sizeof(double));
    s->fE[c] = calloc(s->n1, sizeof(double)); s->fB[c] = calloc(s->n1, sizeof(double));
  }
  s->tmp = calloc(s->n1, sizeof(double));
  s->s_int = calloc(s->n1, sizeof(double));
  s->s_half = calloc(s->n1, sizeof(double));
  for (int k = 0; k <= cfg->nz; k++) {
    s->s_int[k] = pml_sigma(s, (double)k);
    s->s_half[k] = pml_sigma(s, k + 0.5);
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
  s->glo = L + g;
  s->ghi = cfg->nz - L - g;
  s->sp[0].q = -O_QE; s->sp[0].m = O_ME;
  s->sp[1].q = O_QE;  s->sp[1].m = 1836.15267343 * O_ME;
  return s;
}

void o1_destroy(o1_sim* s) {
  if (!s) return;
  for (int c = 0; c < WNCOMP; c++) free(s->F[c]);
  for (int c = 0; c < 3; c++) { free(s->Ep[c]); free(s->Eb[c]); free(s->Ee[c]); free(s->Bold[c]); free(s->fE[c]); free(s->fB[c]); }
  free(s->tmp); free(s->s_int); free(s->s_half);
  for (int q = 0; q < 2; q++) {
    o1_species* p = &s->sp[q];
    free(p->z); free(p->zl); free(p->ux); free(p->uy); free(p->uz); free(p->w); free(p->id); free(p->alive);
  }
  free(s);
}

/* info: dz, dt, gamma, beta, step, t, guard, z_lo, z_hi (cells), z0 */
void o1_info(const o1_sim* s, double* out) {
  out[0] = s->dz; out[1] = s->dt; out[2] = s->gamma; out[3] = s->beta; out[4] = (double)s->step;
  out[5] = time_of(s, s->step); out[6] = s->c.particle_guard; out[7] = s->glo; out[8] = s->ghi; out[9] = s->z0;
}

/* ------------------------------------------------------------------ */
/* Plasma (Sec. 3.1.1, PR-9, PR-12): row m at z'_m(t) = (m + 1/2) h - beta c t, h = dz/ppc_z, density
 * gamma n0(gamma (m + 1/2) h), weight n' dz / ppc_z per unit area; ions fixed in the lab on the same rows. */
static double lab_density(const o1_plasma* p, double zl) {
  if (zl < p->z_start_lab) return 0.0;
  double r = zl - p->z_start_lab;
  if (p->ramp_lab > 0.0 && r < p->ramp_lab) return p->n0 * r / p->ramp_lab;
  double plateau_end = p->ramp_lab + p->length_lab;
  if (p->length_lab > 0.0 && r >= plateau_end) return 0.0;
  return p->n0;
}

static double z_hi_of(const o1_sim* s) { return s->z0 + s->ghi * s->dz; }
static double z_lo_of(const o1_sim* s) { return s->z0 + s->glo * s->dz; }

static long rows_inside(const o1_sim* s, double t) {
  return (long)ceil((z_hi_of(s) + s->beta * O_C * t) / s->h_row - 0.5);
}

static void add_row(o1_sim* s, long m, double t) {
  double zlat = (m + 0.5) * s->h_row;
  double n = s->gamma * lab_density(&s->pl, s->gamma * zlat);
  if (n <= 0.0) return;
  double zp = zlat - s->beta * O_C * t;
  if (zp < z_lo_of(s)) return;
  double w = n * s->dz / (double)s->pl.ppc_z;
  double uz = -s->gamma * s->beta * O_C;
  sp_push(&s->sp[0], zp, 0.0, 0.0, uz, w, (uint32_t)m, zlat);
  if (s->pl.ions) sp_push(&s->sp[1], zp, 0.0, 0.0, uz, w, (uint32_t)m, zlat);
}

int o1_load_plasma(o1_sim* s, const o1_plasma* p) {
  s->pl = *p; s->has_plasma = 1;
  s->h_row = s->dz / p->ppc_z;
  double t = time_of(s, s->step);
  long m_end = rows_inside(s, t);
  long m_beg = (long)ceil((z_lo_of(s) + s->beta * O_C * t) / s->h_row - 0.5);
  for (long m = m_beg; m < m_end; m++) add_row(s, m, t);
  s->row_next = m_end;
  return 0;
}

/* Laser (Sec. 3.1.2): a current sheet at rest at z_antenna emitting the lab waveform
 * E0 exp(-(s - t_peak)^2/(2 sigma^2)) sin(omega (s - t_peak) + phase), s = t'/((1+beta) gamma), with
 * amplitude E0/((1+beta) gamma); K_y = -2 eps0 c E_emit, y-polarised. */
int o1_set_laser(o1_sim* s, const o1_laser* l) {
  s->las = *l; s->has_laser = 1;
  return 0;
}

static double emit_field(const o1_sim* s, double tp) {
  const o1_laser* l = &s->las;
  double om = 2.0 * O_PI * O_C / l->lambda0;
  double E0 = l->a0 * O_ME * O_C * om / O_QE;
  double dop = (1.0 + s->beta) * s->gamma;
  double sl = tp / dop;
  double sig = l->tau_fwhm / (2.0 * sqrt(log(2.0)));
  double g = E0 * exp(-(sl - l->t_peak) * (sl - l->t_peak) / (2.0 * sig * sig)) * sin(om * (sl - l->t_peak) + l->phase);
  return g / dop;
}

static void antenna(o1_sim* s) {
  if (!s->has_laser) return;
  double t0 = time_of(s, s->step), t1 = time_of(s, s->step + 1), th = 0.5 * (t0 + t1);
  double za = s->las.z_antenna;
  if (za < z_lo_of(s) || za >= z_hi_of(s)) return;
  double Z = (za - s->z0) / s->dz;
  int fz = (int)floor(Z);
  double K = -2.0 * O_EPS0 * O_C * emit_field(s, th);
  for (int k = fz - 3; k <= fz + 4; k++) {
    double wz = orc_shape(s->c.order, Z - k);
    if (wz == 0.0 || k < 0 || k > s->c.nz) continue;
    s->F[WJY][k] += K * wz / s->dz;
  }
}

/* ------------------------------------------------------------------ */
static void shift_array(o1_sim* s, double* F, long sh, int comp) {
  int lo, hi;
  vrange(s, comp, &lo, &hi);
  for (int k = 0; k <= s->c.nz; k++) {
    long kk = k + sh;
    double v = kk <= s->c.nz ? F[kk] : 0.0;
    F[k] = (k >= lo && k <= hi) ? v : 0.0;
  }
}

static void window_shift(o1_sim* s) {
  if (!s->c.moving_window) return;
  long want = (long)floor(s->c.window_beta * O_C * time_of(s, s->step) / s->dz);
  long sh = want - s->shifts;
  if (sh <= 0) return;
  for (int c = 0; c < 6; c++) shift_array(s, s->F[c], sh, c);
  for (int c = 0; c < 3; c++) { shift_array(s, s->Ep[c], sh, c); shift_array(s, s->Eb[c], sh, c); }
  s->shifts = want;
  s->z0 = want * s->dz;
}

static void one_step(o1_sim* s) {
  window_shift(s);
  faraday(s);
  for (int c = 0; c < 3; c++)
    for (int k = 0; k < s->n1; k++) {
      s->fE[c][k] = s->F[WEX + c][k];
      s->fB[c][k] = 0.5 * (s->Bold[c][k] + s->F[WBX + c][k]);
    }
  if (s->c.filter_gather)
    for (int c = 0; c < 3; c++) { filter_component(s, WEX + c, s->fE[c]); filter_component(s, WBX + c, s->fB[c]); }
  if (s->c.gather_nodal)
    for (int c = 0; c < 3; c++) { to_nodes(s, WEX + c, s->fE[c]); to_nodes(s, WBX + c, s->fB[c]); }
  for (int c = WJX; c <= WJZ; c++) memset(s->F[c], 0, sizeof(double) * s->n1);
  double zlo = z_lo_of(s), zhi = z_hi_of(s);
  double tn = time_of(s, s->step), tn1 = time_of(s, s->step + 1);
  for (int sp = 0; sp < 2; sp++) {
    o1_species* p = &s->sp[sp];
    for (long q = 0; q < p->n; q++) {
      if (!p->alive[q]) continue;
      double u[3] = { p->ux[q], p->uy[q], p->uz[q] };
      double zn;
      if (sp == 0) {
        double Z = (p->z[q] - s->z0) / s->dz;
        double E[3], B[3];
        for (int c = 0; c < 3; c++) { E[c] = gather1(s, s->fE[c], WEX + c, Z); B[c] = gather1(s, s->fB[c], WBX + c, Z); }
        orc_boris(u, E, B, p->q, p->m, s->dt);
        double gm = sqrt(1.0 + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) / (O_C * O_C));
        zn = p->z[q] + s->dt * u[2] / gm;
        esirkepov1(s, Z, (zn - s->z0) / s->dz, u[0] / gm, u[1] / gm, p->q * p->w[q]);
      } else {
        /* ions fixed in the lab (PR-9) */
        double z0i = p->zl[q] - s->beta * O_C * tn;
        zn = p->zl[q] - s->beta * O_C * tn1;
        esirkepov1(s, (z0i - s->z0) / s->dz, (zn - s->z0) / s->dz, 0.0, 0.0, p->q * p->w[q]);
      }
      p->z[q] = zn;
      p->ux[q] = u[0]; p->uy[q] = u[1]; p->uz[q] = u[2];
      if (zn < zlo || zn >= zhi + s->dz) p->alive[q] = 0;
    }
  }
  antenna(s);
  if (s->c.filter_J) for (int c = 0; c < 3; c++) filter_component(s, WJX + c, s->F[WJX + c]);
  ampere(s);
  sp_compact(&s->sp[0]); sp_compact(&s->sp[1]);
  s->step++;
  if (s->has_plasma) {
    double t = time_of(s, s->step);
    long m_end = rows_inside(s, t);
    for (long m = s->row_next; m < m_end; m++) add_row(s, m, t);
    if (m_end > s->row_next) s->row_next = m_end;
  }
}

int o1_step(o1_sim* s, int n) {
  for (int i = 0; i < n; i++) one_step(s);
  return 0;
}

void o1_get_field(const o1_sim* s, int comp, double* out) { memcpy(out, s->F[comp], sizeof(double) * s->n1); }
void o1_set_field(o1_sim* s, int comp, const double* in) { memcpy(s->F[comp], in, sizeof(double) * s->n1); }
void o1_get_gather_field(const o1_sim* s, int comp, double* out) {
  memcpy(out, comp < 3 ? s->fE[comp] : s->fB[comp - 3], sizeof(double) * s->n1);
}
long o1_num_particles(const o1_sim* s, int species) { return s->sp[species].n; }

/* replaces the particles of a species (test input; ids 0..n-1; an ion keeps z as its lab row) */
void o1_set_particles(o1_sim* s, int species, long n, const double* z, const double* ux, const double* uy,
                      const double* uz, const double* w) {
  o1_species* p = &s->sp[species];
  p->n = 0;
  for (long j = 0; j < n; j++) sp_push(p, z[j], ux[j], uy[j], uz[j], w[j], (uint32_t)j, z[j]);
}
void o1_get_particles(const o1_sim* s, int species, double* z, double* ux, double* uy, double* uz, double* w,
                      uint32_t* id) {
  const o1_species* p = &s->sp[species];
  for (long j = 0; j < p->n; j++) {
    z[j] = p->z[j]; ux[j] = p->ux[j]; uy[j] = p->uy[j]; uz[j] = p->uz[j]; w[j] = p->w[j]; id[j] = p->id[j];
  }
}

/* charge density at the nodes (both species), the shape of the run's order */
void o1_rho(const o1_sim* s, double* rho) {
  memset(rho, 0, sizeof(double) * s->n1);
  for (int sp = 0; sp < 2; sp++) {
    const o1_species* p = &s->sp[sp];
    for (long q = 0; q < p->n; q++) {
      double Z = (p->z[q] - s->z0) / s->dz;
      int f = (int)floor(Z);
      for (int k = f - 3; k <= f + 3; k++) {
        double wz = orc_shape(s->c.order, Z - k);
        if (wz != 0.0 && k >= 0 && k <= s->c.nz) rho[k] += p->q * p->w[q] * wz / s->dz;
      }
    }
  }
}

/* diagnostics: [0] electrons, [1] field energy per unit area (eps0 E^2 + B^2/mu0)/2 dz summed */
void o1_diag(const o1_sim* s, double* out) {
  double en = 0.0;
  for (int k = 0; k < s->n1; k++) {
    double e2 = 0.0, b2 = 0.0;
    for (int c = 0; c < 3; c++) { e2 += s->F[WEX + c][k] * s->F[WEX + c][k]; b2 += s->F[WBX + c][k] * s->F[WBX + c][k]; }
    en += 0.5 * (O_EPS0 * e2 + b2 / O_MU0) * s->dz;
  }
  out[0] = (double)s->sp[0].n;
  out[1] = en;
}
