// Auxiliary kernels of the boosted-frame PIC step:
//  - the current of the ions fixed in the lab (PR-9): they move rigidly at
//    -beta c on the electrons' lattice, so the sum of their Esirkepov currents
//    factorises into a transverse lattice profile times a per-column prefix
//    sum of the change of the deposited row density (exact, no particles);
//  - the laser antenna current (Sec. 3.1.2, PR-13/14);
//  - the test beam through a plane (Sec. 3.1.1): Lorentz transform and push;
//  - back-transformed lab-frame samples (Sec. 3.2, PR-16);
//  - charge density, reductions, moving-window shift, copies.

#include "../../include/pic.h"
#include "pic_common.cuh"

namespace picgb {

namespace {

__device__ __forceinline__ double shape_val(int order, double s) {
  double a = fabs(s);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { double t = 2.0 - a; return t * t * t / 6.0; }
  return 0.0;
}

__device__ double lab_density_d(const InjectP& ip, double zl) {
  if (zl < ip.z_start_lab) return 0.0;
  double r = zl - ip.z_start_lab;
  if (ip.ramp_lab > 0.0 && r < ip.ramp_lab) return ip.n0 * r / ip.ramp_lab;
  double pe = ip.ramp_lab + ip.length_lab;
  if (ip.length_lab > 0.0 && r >= pe) return 0.0;
  return ip.n0;
}

// R(k) = sum over live rows of w_m S(Z_m(t) - k) at two times (blockIdx.y selects the time):
// the row density of the rigid ions, for their charge density
__global__ void k_ion_rows(GridP g, long long mlo, long long mhi, double t0, double t1, InjectP ip, int order,
                           double* R0, double* R1) {
  // one warp per (node k, time); the lanes stride over the lattice rows within the shape's reach
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k > g.nz) return;   // uniform over the warp
  const double reach = order == 3 ? 2.0 : 1.0;
  const double wfac = g.dx * g.dz / (double)(ip.ppc_x * ip.ppc_z);
  const double t = blockIdx.y == 0 ? t0 : t1;
  const double shift = ip.beta * kC * t;
  long long ma = (long long)floor(((k - reach) * g.dz + g.z0 + shift) / ip.h - 0.5) - 1;
  long long mb = (long long)ceil(((k + reach) * g.dz + g.z0 + shift) / ip.h - 0.5) + 1;
  if (ma < mlo) ma = mlo;
  if (mb > mhi - 1) mb = mhi - 1;
  double acc = 0.0;
  for (long long m = ma + lane; m <= mb; m += 32) {
    const double zlat = (m + 0.5) * ip.h;
    const double Zm = (zlat - shift - g.z0) / g.dz;
    const double sv = shape_val(order, Zm - k);
    if (sv == 0.0) continue;
    acc += ip.gamma * lab_density_d(ip, ip.gamma * zlat) * wfac * sv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) (blockIdx.y == 0 ? R0 : R1)[k] = acc;
}

// Column current of the rigid ions (PR-9): a lattice row m of line density n_m
// moving from Z0 to Z1 (in cells) during the step carries through the face
// above node k the charge n_m [CS(Z1, k) - CS(Z0, k)], with CS(Z, k) the sum of
// the row's shape weights on the nodes <= k (the 1D Esirkepov current). One
// thread per row adds its non-zero terms (at most NG+1 nodes) to C.
__device__ __forceinline__ double cum_weight(int order, double Z, int k) {
  const int fz = (int)floor(Z);
  const double t = Z - fz;
  const int off = order == 3 ? 1 : 0;
  const int j = k - (fz - off);   // index of node k in the row's stencil
  if (j < 0) return 0.0;
  if (order == 3) {
    if (j >= 3) return 1.0;
    const double t2 = t * t, t3 = t2 * t, s = 1.0 - t;
    const double w0 = s * s * s * (1.0 / 6.0);
    if (j == 0) return w0;
    const double w1 = 2.0 / 3.0 - t2 + 0.5 * t3;
    if (j == 1) return w0 + w1;
    return 1.0 - t3 * (1.0 / 6.0);
  }
  return j >= 1 ? 1.0 : 1.0 - t;
}

__global__ void k_ion_current(GridP g, long long mlo, long long mhi, double t0, double t1, InjectP ip, int order,
                              double* C) {
  const long long m = mlo + (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= mhi) return;
  const double wfac = g.dx * g.dz / (double)(ip.ppc_x * ip.ppc_z);
  const double zlat = (m + 0.5) * ip.h;
  const double nm = ip.gamma * lab_density_d(ip, ip.gamma * zlat) * wfac;
  if (nm == 0.0) return;
  const double Z0 = (zlat - ip.beta * kC * t0 - g.z0) / g.dz;
  const double Z1 = (zlat - ip.beta * kC * t1 - g.z0) / g.dz;
  const int off = order == 3 ? 1 : 0, ng = order == 3 ? 4 : 2;
  const int klo = (int)floor(fmin(Z0, Z1)) - off;
  const int khi = (int)floor(fmax(Z0, Z1)) - off + ng - 2;
  for (int k = max(klo, 0); k <= min(khi, g.nz); k++) {
    const double d = cum_weight(order, Z1, k) - cum_weight(order, Z0, k);
    if (d != 0.0) atomicAdd(&C[k], nm * d);
  }
}

// ---------------------------------------------------------------------------
// antenna: J_y of one +/- pair per transverse node (Sec. 3.1.2). The emitted
// field factorises into a time factor (amp) and the transverse Gaussian; xs[i]
// is that Gaussian already weighted by the x shape, and wz[] the z weights of
// the antenna's positions at t^n and t^{n+1}, averaged and divided by dz.
template <class T>
__global__ void k_antenna(GridP g, T* Jy, const double* xs, AntennaStep a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > g.nx) return;
  const double kx = a.amp * xs[i];
  if (kx == 0.0) return;
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int k = a.k0 + j;
    if (a.wz[j] != 0.0 && k >= 0 && k <= g.nz) Jy[(long)i * g.ld + k] += T(kx * a.wz[j]);
  }
}

// ---------------------------------------------------------------------------
// test beam through a plane (Sec. 3.1.1, Eq. t*..Eq. zp)
__global__ void k_beam_sum_vz(int n, const double* ux, const double* uy, const double* uz, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double gj = sqrt(1.0 + (ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) / (kC * kC));
  atomicAdd(&acc[0], uz[j] / gj);
}

template <class T>
__global__ void k_beam_transform(Beam<T> b, const double* lx, const double* lz, const double* lux, const double* luy,
                                 const double* luz, double t_lab, double z_plane, double gam, double be, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  const double betab = acc[0] / b.n / kC;
  const double gj = sqrt(1.0 + (lux[j] * lux[j] + luy[j] * luy[j] + luz[j] * luz[j]) / (kC * kC));
  const double vx = lux[j] / gj, vy = luy[j] / gj, vz = luz[j] / gj;
  const double tcross = t_lab + (z_plane - lz[j]) / vz;
  const double xs = lx[j] + vx * (tcross - t_lab);
  const double tpc = gam * (tcross - be * z_plane / kC);
  const double zpc = gam * (z_plane - be * kC * tcross);
  const double den = 1.0 - be * betab;
  const double vxp = vx / (gam * den), vyp = vy / (gam * den), vzp = (vz - be * kC) / den;
  const double v2 = (vxp * vxp + vyp * vyp + vzp * vzp) / (kC * kC);
  const double gp = 1.0 / sqrt(1.0 - v2);
  b.x[j] = xs;
  b.uxb[j] = T(gp * vxp); b.uyb[j] = T(gp * vyp); b.uzb[j] = T(gp * vzp);
  b.ux[j] = b.uxb[j]; b.uy[j] = b.uyb[j]; b.uz[j] = b.uzb[j];
  b.tc[j] = tpc;
  b.zf0[j] = zpc;   // completed by k_beam_finish
  b.flag[j] = 1;    // alive, frozen
  atomicAdd(&acc[1], vzp);
}

template <class T>
__global__ void k_beam_finish(Beam<T> b, double t_now, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  const double vbar = acc[1] / b.n;
  const double zf = b.zf0[j] - vbar * b.tc[j];
  b.zf0[j] = zf;
  b.z[j] = zf + vbar * t_now;
  if (j == 0) acc[2] = vbar;
}

template <class T>
__device__ T gather_global(const T* F, const GridP& g, int order, double X, double Z, double sx, double sz) {
  const int fx = (int)floor(X), fz = (int)floor(Z);
  double acc = 0.0;
  for (int i = fx - 3; i <= fx + 3; i++) {
    const double wx = shape_val(order, X - (i + sx));
    if (wx == 0.0 || i < 0 || i > g.nx) continue;
    for (int k = fz - 3; k <= fz + 3; k++) {
      const double wz = shape_val(order, Z - (k + sz));
      if (wz == 0.0 || k < 0 || k > g.nz) continue;
      acc += (double)F[(long)i * g.ld + k] * wx * wz;
    }
  }
  return T(acc);
}

// Esirkepov deposit of one beam particle (charge * weight qw per unit length along y) moving (x0, z0) ->
// (x1, z1) with out-of-plane velocity vy, into the global current with atomics (a beam has few particles):
// Jx(i+1/2) - Jx(i-1/2) = -qw/(dz dt) Wx(i), Wx = DSx (S0z + DSz/2); likewise for Jz; Jy = qw vy Wy/(dx dz),
// Wy = S0x S0z + DSx S0z/2 + S0x DSz/2 + DSx DSz/3 (Esirkepov 2001)
template <class T>
__device__ void beam_deposit(const GridP& g, const FieldPtrs<T>& f, int order, double x0, double z0, double x1,
                             double z1, double vy, double qw) {
  constexpr int EW = 9;
  const double X0 = x0 / g.dx, Z0 = (z0 - g.z0) / g.dz, X1 = x1 / g.dx, Z1 = (z1 - g.z0) / g.dz;
  const int bx = (int)floor(X0 < X1 ? X0 : X1) - 3, bz = (int)floor(Z0 < Z1 ? Z0 : Z1) - 3;
  double S0x[EW], DSx[EW], S0z[EW], DSz[EW];
  for (int a = 0; a < EW; a++) {
    S0x[a] = shape_val(order, X0 - (bx + a));
    DSx[a] = shape_val(order, X1 - (bx + a)) - S0x[a];
    S0z[a] = shape_val(order, Z0 - (bz + a));
    DSz[a] = shape_val(order, Z1 - (bz + a)) - S0z[a];
  }
  const double cx = -qw / (g.dz * g.dt), cz = -qw / (g.dx * g.dt), cy = qw * vy / (g.dx * g.dz);
  for (int b = 0; b < EW; b++) {
    double acc = 0.0;
    for (int a = 0; a < EW; a++) {
      acc += cx * DSx[a] * (S0z[b] + 0.5 * DSz[b]);
      const int i = bx + a, k = bz + b;
      if (acc != 0.0 && i >= 0 && i <= g.nx && k >= 0 && k <= g.nz) atomicAdd(f.J[0] + (long)i * g.ld + k, T(acc));
    }
  }
  for (int a = 0; a < EW; a++) {
    double acc = 0.0;
    for (int b = 0; b < EW; b++) {
      acc += cz * DSz[b] * (S0x[a] + 0.5 * DSx[a]);
      const int i = bx + a, k = bz + b;
      if (acc != 0.0 && i >= 0 && i <= g.nx && k >= 0 && k <= g.nz) atomicAdd(f.J[2] + (long)i * g.ld + k, T(acc));
    }
  }
  if (vy != 0.0)
    for (int a = 0; a < EW; a++)
      for (int b = 0; b < EW; b++) {
        const double wy = S0x[a] * S0z[b] + 0.5 * DSx[a] * S0z[b] + 0.5 * S0x[a] * DSz[b] + DSx[a] * DSz[b] / 3.0;
        const int i = bx + a, k = bz + b;
        if (wy != 0.0 && i >= 0 && i <= g.nx && k >= 0 && k <= g.nz)
          atomicAdd(f.J[1] + (long)i * g.ld + k, T(cy * wy));
      }
}

template <class T>
__device__ __forceinline__ void beam_push_one(const GridP& g, const FieldPtrs<T>& f, const Beam<T>& b, int order,
                                              double tn, double tn1, int nodal, const double* acc, int j) {
  int fl = b.flag[j];
  if (!(fl & 1)) return;
  const double xlo = g.gx_lo * g.dx, xhi = g.gx_hi * g.dx;
  const double zlo = g.z0 + g.gz_lo * g.dz, zhi = g.z0 + g.gz_hi * g.dz + g.dz;
  if (!(fl & 2)) {
    if (tn >= b.tc[j]) {
      fl |= 2;
      b.ux[j] = b.uxb[j]; b.uy[j] = b.uyb[j]; b.uz[j] = b.uzb[j];
      // a particle whose crossing lies outside the particle domain never enters it (PR-20)
      const double xa = b.x[j], za = b.z[j];
      if (xa < xlo || xa >= xhi || za < zlo || za >= zhi) fl &= ~1;
      b.flag[j] = fl;
      if (!(fl & 1)) return;
    } else {
      const double z0 = b.z[j], z1 = b.zf0[j] + acc[2] * tn1, x0 = b.x[j];
      // self-consistent beam: a frozen particle inside the particle domain carries its charge along z
      if (b.self && x0 >= xlo && x0 < xhi && z0 >= zlo && z0 < zhi && z1 >= zlo && z1 < zhi)
        beam_deposit<T>(g, f, order, x0, z0, x0, z1, 0.0, -kQe * (double)b.w[j]);
      b.z[j] = z1;
      return;
    }
  }
  const double x = b.x[j], z = b.z[j];
  const double X = x / g.dx, Z = (z - g.z0) / g.dz;
  // Yee locations, or the node values of the 'momentum conserving' gather (offsets 0)
  const double h = nodal ? 0.0 : 0.5;
  const T* const* gE = nodal ? f.nE : f.fE;
  const T* const* gB = nodal ? f.nB : f.fB;
  const double E[3] = {(double)gather_global<T>(gE[0], g, order, X, Z, h, 0.0),
                       (double)gather_global<T>(gE[1], g, order, X, Z, 0.0, 0.0),
                       (double)gather_global<T>(gE[2], g, order, X, Z, 0.0, h)};
  const double B[3] = {(double)gather_global<T>(gB[0], g, order, X, Z, 0.0, h),
                       (double)gather_global<T>(gB[1], g, order, X, Z, h, h),
                       (double)gather_global<T>(gB[2], g, order, X, Z, h, 0.0)};
  const T k = T(-kQe * g.dt / (2.0 * kMe));
  const T ic2 = T(1.0 / (kC * kC));
  T ux = b.ux[j], uy = b.uy[j], uz = b.uz[j];
  T umx = ux + k * T(E[0]), umy = uy + k * T(E[1]), umz = uz + k * T(E[2]);
  T gm = sqrt(T(1) + (umx * umx + umy * umy + umz * umz) * ic2);
  T tbx = k * T(B[0]) / gm, tby = k * T(B[1]) / gm, tbz = k * T(B[2]) / gm;
  T t2 = tbx * tbx + tby * tby + tbz * tbz;
  T sf = T(2) / (T(1) + t2);
  T upx = umx + (umy * tbz - umz * tby), upy = umy + (umz * tbx - umx * tbz), upz = umz + (umx * tby - umy * tbx);
  T plx = umx + sf * (upy * tbz - upz * tby), ply = umy + sf * (upz * tbx - upx * tbz),
    plz = umz + sf * (upx * tby - upy * tbx);
  ux = plx + k * T(E[0]); uy = ply + k * T(E[1]); uz = plz + k * T(E[2]);
  const T g1 = sqrt(T(1) + (ux * ux + uy * uy + uz * uz) * ic2);
  const double xn = x + g.dt * (double)(ux / g1);
  const double zn = z + g.dt * (double)(uz / g1);
  if (b.self) beam_deposit<T>(g, f, order, x, z, xn, zn, (double)(uy / g1), -kQe * (double)b.w[j]);
  b.x[j] = xn; b.z[j] = zn; b.ux[j] = ux; b.uy[j] = uy; b.uz[j] = uz;
  if (xn < xlo || xn >= xhi || zn < zlo || zn >= zhi) b.flag[j] = fl & ~1;
}

template <class T>
__global__ void k_beam_push(GridP g, FieldPtrs<T> f, Beam<T> b, int order, double tn, double tn1, int nodal,
                            const double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  beam_push_one<T>(g, f, b, order, tn, tn1, nodal, acc, j);
}

// the batched step's test beams: run blockIdx.y, its particles from blockIdx.x * 128 (the Yee-located
// gather; the batched step carries no node-interpolated runs)
template <class T>
__global__ void k_beam_push_batch(const StepArgs<T>* a) {
  const StepArgs<T>& A = a[blockIdx.y];
  if (!A.beam_on) return;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= A.beam.n) return;
  beam_push_one<T>(A.g, A.f, A.beam, A.beam_order, A.beam_tn, A.beam_tn1, 0, A.beam_acc, j);
}

// ---------------------------------------------------------------------------
// back-transformed samples: rows [r0, r1) of the t'-sorted list
template <class T>
__device__ double interp_z(const T* F, const GridP& g, int i, double zp, double stz) {
  const double Z = (zp - g.z0) / g.dz - stz;
  const int k = (int)floor(Z);
  const double fr = Z - k;
  double a = 0.0, b = 0.0;
  if (k >= 0 && k <= g.nz) a = (double)F[(long)i * g.ld + k];
  if (k + 1 >= 0 && k + 1 <= g.nz) b = (double)F[(long)i * g.ld + k + 1];
  return (1.0 - fr) * a + fr * b;
}

template <class T>
__global__ void k_btd(GridP g, FieldPtrs<T> f, int which, int post, int r0, int r1, const int* order_idx,
                      const double* tp, const double* zp, double ta, double gam, double be, T* out, int* done) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int rr = r0 + blockIdx.y;
  if (rr >= r1 || i > g.nx) return;
  const int row = order_idx[rr];
  const double fr = (tp[rr] - ta) / g.dt;
  const double wgt = post ? fr : 1.0 - fr;
  const double z = zp[rr];
  const int nxp = g.nx + 1;
  T* o = out + (size_t)row * 6 * nxp;
  if (which == 0) {
    const double ex = interp_z<T>(f.E[0], g, i, z, 0.0);
    const double ey = interp_z<T>(f.E[1], g, i, z, 0.0);
    const double ez = interp_z<T>(f.E[2], g, i, z, 0.5);
    o[0 * nxp + i] += T(wgt * gam * ex);
    o[1 * nxp + i] += T(wgt * gam * ey);
    o[2 * nxp + i] += T(wgt * ez);
    o[3 * nxp + i] += T(wgt * (-gam * be * ey / kC));
    o[4 * nxp + i] += T(wgt * (gam * be * ex / kC));
  } else {
    const double bx = interp_z<T>(f.B[0], g, i, z, 0.5);
    const double by = interp_z<T>(f.B[1], g, i, z, 0.5);
    const double bz = interp_z<T>(f.B[2], g, i, z, 0.0);
    o[0 * nxp + i] += T(wgt * gam * be * kC * by);
    o[1 * nxp + i] += T(wgt * (-gam * be * kC * bx));
    o[3 * nxp + i] += T(wgt * gam * bx);
    o[4 * nxp + i] += T(wgt * gam * by);
    o[5 * nxp + i] += T(wgt * bz);
  }
  if (post && i == 0) done[2 * row + which] = 1;
}

// ---------------------------------------------------------------------------
template <class T>
__global__ void k_rho(GridP g, Particles<T> p, const Ctrl* ctrl, int order, double q, double* rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->count) return;
  const double w = (double)p.w[j];
  if (!(w > 0.0)) return;   // ghosts (negative weight) are ions, counted by the ion charge density
  double X, Z;
  if constexpr (CellPos<T>::value) {
    int iz;
    float tz;
    frame_z(p.cell[j], p.oz[j], g.fr_sz, g.fr_fz, iz, tz);
    X = cell_x(p.cell[j]) + (double)p.ox[j];
    Z = iz + (double)tz;
  } else {
    X = p.x[j] / g.dx; Z = (p.z[j] - g.z0) / g.dz;
  }
  const int fx = (int)floor(X), fz = (int)floor(Z);
  for (int i = fx - 2; i <= fx + 3; i++)
    for (int k = fz - 2; k <= fz + 3; k++) {
      const double s = shape_val(order, X - i) * shape_val(order, Z - k);
      if (s != 0.0 && i >= 0 && i <= g.nx && k >= 0 && k <= g.nz)
        atomicAdd(&rho[(long)i * (g.nz + 1) + k], q * w * s / (g.dx * g.dz));
    }
}

__global__ void k_ion_rho(GridP g, const double* ion_x, const double* R, double coef, double* rho) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (k > g.nz) return;
  rho[(long)i * (g.nz + 1) + k] += coef * ion_x[i] * R[k];
}

template <class T>
__global__ void __launch_bounds__(256) k_stats(GridP g, FieldPtrs<T> f, Particles<T> p, const Ctrl* ctrl, Beam<T> b,
                                               double gam, double be, double trap, double* out) {
  // out: [0] n_e, [1] n_beam_active, [2] sum gamma_lab, [3] sum gamma_lab^2, [4] field energy,
  // [5] weight of the electrons with lab-frame gamma above trap
  __shared__ double red[6][256];
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthr = (long)gridDim.x * blockDim.x;
  double ne = 0, na = 0, sg = 0, sg2 = 0, en = 0, wt = 0;
  const int nz1 = g.nz + 1;
  const int ncell = (g.nx + 1) * nz1;
  if (sizeof(T) == 4) {
    // FP32 path (momenta and fields in FP32): the lab-gamma test and the per-thread sums (a few dozen
    // particles, a few nodes) in FP32, the block and grid sums in FP64; the FP64 pipe of this GPU is narrow
    const float ic2 = float(1.0 / (kC * kC)), ic = float(1.0 / kC);
    const float gamf = float(gam), bef = float(be), trapf = float(trap);
    int nef = 0;
    float wtf = 0.f;
    const long n = ctrl->count;
    if (trap > 0.0) {
      // four consecutive particles per iteration from 16-byte loads of each array (the arrays are 16-byte
      // aligned), every load of an iteration issued at once, two iterations in flight; the last n % 4
      // particles one by one
      auto one = [&](float w, float ux, float uy, float uzs) {
        // boosted-frame momentum (the mixed path stores u_z - u0) -> lab-frame gamma
        const float uz = CellPos<T>::value ? g.fr_u0 + uzs : uzs;
        const bool live = w > 0.f;
        nef += live ? 1 : 0;
        const float gp = sqrtf(1.f + (ux * ux + uy * uy + uz * uz) * ic2);
        if (live && gamf * (gp + bef * uz * ic) > trapf) wtf += w;
      };
      // (arrays from an allocator that does not align to 16 bytes take the one-by-one loop throughout)
      const bool al16 = ((reinterpret_cast<uintptr_t>(p.w) | reinterpret_cast<uintptr_t>(p.ux) |
                          reinterpret_cast<uintptr_t>(p.uy) | reinterpret_cast<uintptr_t>(p.uz)) & 15) == 0;
      const long n4 = al16 ? n / 4 : 0;
      const float4* w4 = reinterpret_cast<const float4*>(p.w);
      const float4* x4 = reinterpret_cast<const float4*>(p.ux);
      const float4* y4 = reinterpret_cast<const float4*>(p.uy);
      const float4* z4 = reinterpret_cast<const float4*>(p.uz);
#pragma unroll 2
      for (long j = tid; j < n4; j += nthr) {
        const float4 w = w4[j], ux = x4[j], uy = y4[j], uz = z4[j];
        one(w.x, ux.x, uy.x, uz.x);
        one(w.y, ux.y, uy.y, uz.y);
        one(w.z, ux.z, uy.z, uz.z);
        one(w.w, ux.w, uy.w, uz.w);
      }
      for (long j = 4 * n4 + tid; j < n; j += nthr) one(float(p.w[j]), float(p.ux[j]), float(p.uy[j]), float(p.uz[j]));
    } else {
#pragma unroll 4
      for (long j = tid; j < n; j += nthr) nef += float(p.w[j]) > 0.f ? 1 : 0;
    }
    ne = nef;
    wt = wtf;
    const float e0 = float(kEps0), imu0 = float(kEps0 * kC * kC);
    float enf = 0.f;
#pragma unroll 4
    for (int e = (int)tid; e < ncell; e += (int)nthr) {
      const int i = e / nz1, k = e - i * nz1;
      const long q = (long)i * g.ld + k;
      float e2 = 0.f, b2 = 0.f;
      for (int c = 0; c < 3; c++) {
        const float ev = float(f.E[c][q]), bv = float(f.B[c][q]);
        e2 += ev * ev; b2 += bv * bv;
      }
      enf += e0 * e2 + b2 * imu0;
    }
    en = 0.5 * (double)enf * g.dx * g.dz;
  } else {
    for (long j = tid; j < ctrl->count; j += nthr) {
      const double w = (double)p.w[j];
      if (!(w > 0.0)) continue;
      ne += 1.0;
      if (trap > 0.0) {
        const double ux = p.ux[j], uy = p.uy[j];
        const double uz = CellPos<T>::value ? (double)g.fr_u0 + (double)p.uz[j] : (double)p.uz[j];
        const double gp = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
        if (gam * (gp + be * uz / kC) > trap) wt += w;
      }
    }
    const double mu0 = 1.0 / (kEps0 * kC * kC);
    for (int e = (int)tid; e < ncell; e += (int)nthr) {
      const int i = e / nz1, k = e - i * nz1;
      const long q = (long)i * g.ld + k;
      double e2 = 0, b2 = 0;
      for (int c = 0; c < 3; c++) {
        const double ev = f.E[c][q], bv = f.B[c][q];
        e2 += ev * ev; b2 += bv * bv;
      }
      en += 0.5 * (kEps0 * e2 + b2 / mu0) * g.dx * g.dz;
    }
  }
  for (long j = tid; j < b.n; j += nthr) {
    if ((b.flag[j] & 3) != 3) continue;
    const double ux = b.ux[j], uy = b.uy[j], uz = b.uz[j];
    const double gp = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
    const double gl = gam * (gp + be * uz / kC);
    na += 1; sg += gl; sg2 += gl * gl;
  }
  red[0][threadIdx.x] = ne; red[1][threadIdx.x] = na; red[2][threadIdx.x] = sg;
  red[3][threadIdx.x] = sg2; red[4][threadIdx.x] = en; red[5][threadIdx.x] = wt;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 6; c++) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; c++) atomicAdd(&out[c], red[c][0]);
}

template <class T>
__global__ void k_shift_copy(GridP g, const T* src, T* dst, int sh, int comp) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (k > g.nz) return;
  int i0, i1, k0, k1;
  valid_range(comp, g.nx, g.nz, i0, i1, k0, k1);
  // the PEC walls move with the grid: values stay on the component's valid range
  const bool v = i >= i0 && i <= i1 && k >= k0 && k <= k1;
  dst[(long)i * g.ld + k] = (v && k + sh <= g.nz) ? src[(long)i * g.ld + k + sh] : T(0);
}

__global__ void k_shift_chunks(Chunk* c, const Ctrl* ctrl, int sh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->nchunks) return;
  if (c[j].ix0 <= c[j].ix1) { c[j].iz0 -= sh; c[j].iz1 -= sh; }
}

template <class T>
__global__ void k_convert(const T* src, double* dst, GridP g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (k > g.nz) return;
  dst[(long)i * (g.nz + 1) + k] = (double)src[(long)i * g.ld + k];
}

template <class T>
__global__ void k_convert_back(const double* src, T* dst, GridP g) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  if (k > g.nz) return;
  dst[(long)i * g.ld + k] = T(src[(long)i * (g.nz + 1) + k]);
}

template <class T>
__global__ void k_compact(GridP g, Particles<T> p, const Ctrl* ctrl, double* out6, uint32_t* ido, int* nout,
                          int cap_out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->count) return;
  if (!(p.w[j] > T(0))) return;   // electrons only (ghosts carry ions)
  const int o = atomicAdd(nout, 1);
  if (o >= cap_out) return;
  if constexpr (CellPos<T>::value) {
    int iz;
    float tz;
    frame_z(p.cell[j], p.oz[j], g.fr_sz, g.fr_fz, iz, tz);
    out6[0 * (size_t)cap_out + o] = (cell_x(p.cell[j]) + (double)p.ox[j]) * g.dx;
    out6[1 * (size_t)cap_out + o] = g.z0 + (iz + (double)tz) * g.dz;
  } else {
    out6[0 * (size_t)cap_out + o] = p.x[j];
    out6[1 * (size_t)cap_out + o] = p.z[j];
  }
  out6[2 * (size_t)cap_out + o] = p.ux[j];
  out6[3 * (size_t)cap_out + o] = p.uy[j];
  out6[4 * (size_t)cap_out + o] = CellPos<T>::value ? (double)g.fr_u0 + (double)p.uz[j] : (double)p.uz[j];
  out6[5 * (size_t)cap_out + o] = p.w[j];
  if constexpr (CellPos<T>::value) {
    // stored (row << kb) | column -> row * nxl + column
    const uint32_t id = p.id[j];
    ido[o] = (id >> g.il_kb) * (uint32_t)g.il_nxl + (id & ((1u << g.il_kb) - 1u));
  } else {
    ido[o] = p.id[j];
  }
}

// moving window: the stored cells of the mixed path move with the grid
template <class T>
__global__ void k_shift_particles(GridP g, Particles<T> p, const Ctrl* ctrl, int sh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->count) return;
  if (p.w[j] == T(0)) return;
  const uint32_t c = p.cell[j];
  int iz;
  float tz;
  if (p.w[j] < T(0)) {   // ghost: its lab-fixed ion (g.z0_cells is the origin before this shift)
    uint32_t cs;
    float ox, oz;
    const uint32_t id = p.id[j];
    lattice_site((int)(id >> g.il_kb), (int)(id & ((1u << g.il_kb) - 1u)), g.il_ppcx, g.il_ppcz, g.gx_lo,
                 g.z0_cells, cs, ox, oz);
    frame_z(cs, oz, g.fr_sz, g.fr_fz, iz, tz);
    if (iz - sh < 0) p.w[j] = T(0);
    return;
  }
  frame_z(c, p.oz[j], g.fr_sz, g.fr_fz, iz, tz);
  if (iz - sh < 0) { p.w[j] = T(0); return; }
  p.cell[j] = pack_cell(cell_x(c), (cell_z(c) - sh) & 0xffff);
}

// batched antenna (each run's blocks also clear its ion-column sums for the next kernel)
template <class T>
__global__ void k_antenna_batch(const StepArgs<T>* a, const int* off, int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0) s_r = batch_run(off, nruns, blockIdx.x);
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  const int lb = blockIdx.x - off[s_r], nb = off[s_r + 1] - off[s_r];
  if (A.ion_on)
    for (int k = lb * blockDim.x + threadIdx.x; k <= A.g.nz; k += nb * blockDim.x) A.ion_C[k] = 0.0;
  if (!A.ant_on) return;
  const int i = lb * blockDim.x + threadIdx.x;
  if (i > A.g.nx) return;
  const double kx = A.ast.amp * A.ant_xs[i];
  if (kx == 0.0) return;
  T* Jy = A.f.J[1];
#pragma unroll
  for (int j = 0; j < 8; j++) {
    const int k = A.ast.k0 + j;
    if (A.ast.wz[j] != 0.0 && k >= 0 && k <= A.g.nz) Jy[(long)i * A.g.ld + k] += T(kx * A.ast.wz[j]);
  }
}

// batched rigid-ion column current: rows [ion_mlo, ion_mhi) of each run, one thread per row
template <class T>
__global__ void k_ion_current_batch(const StepArgs<T>* a, const int* off, int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0) s_r = batch_run(off, nruns, blockIdx.x);
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  if (!A.ion_on) return;
  const long long m = A.ion_mlo + (long long)(blockIdx.x - off[s_r]) * blockDim.x + threadIdx.x;
  if (m >= A.ion_mhi) return;
  const GridP& g = A.g;
  const InjectP& ip = A.ip;
  const double wfac = g.dx * g.dz / (double)(ip.ppc_x * ip.ppc_z);
  const double zlat = (m + 0.5) * ip.h;
  const double nm = ip.gamma * lab_density_d(ip, ip.gamma * zlat) * wfac;
  if (nm == 0.0) return;
  const double Z0 = (zlat - ip.beta * kC * A.ion_t0 - g.z0) / g.dz;
  const double Z1 = (zlat - ip.beta * kC * A.ion_t1 - g.z0) / g.dz;
  const int ord = A.ion_order;
  const int o = ord == 3 ? 1 : 0, ng = ord == 3 ? 4 : 2;
  const int klo = (int)floor(fmin(Z0, Z1)) - o;
  const int khi = (int)floor(fmax(Z0, Z1)) - o + ng - 2;
  for (int k = max(klo, 0); k <= min(khi, g.nz); k++) {
    const double d = cum_weight(ord, Z1, k) - cum_weight(ord, Z0, k);
    if (d != 0.0) atomicAdd(&A.ion_C[k], nm * d);
  }
}

}  // namespace

template <class T>
void launch_antenna_ion_batch(const StepArgs<T>* a, const BatchGrid& bg, bool any_ion, cudaStream_t s) {
  k_antenna_batch<T><<<bg.ant_blocks, 128, 0, s>>>(a, bg.ant_off, bg.nruns);
  if (any_ion) k_ion_current_batch<T><<<bg.ion_blocks, 256, 0, s>>>(a, bg.ion_off, bg.nruns);
}

// ---------------------------------------------------------------------------
// Charge density without device allocation: the ion row density R(k) goes to
// this file-scope scratch instead of a context buffer. Its device address is
// looked up on every call, with the caller's device current: the lookup
// allocates nothing, and a cached address could go stale if the caller reset
// the device and the module were loaded again elsewhere.
static __device__ __align__(256) double g_noalloc_rows[PIC_NOALLOC_MAX_NZ + 1];

template <class T>
int launch_rho_noalloc(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int order, bool ions,
                       long long mlo, long long mhi, double t, const InjectP& ip, const double* ion_x, double* dst,
                       cudaStream_t s, cudaError_t* why, int* kernels) {
  *why = cudaSuccess;
  *kernels = 0;
  if (g.nz > PIC_NOALLOC_MAX_NZ) return 1;
  // a launch error left on this thread by unrelated work is not this call's failure
  (void)cudaGetLastError();
  void* addr = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_rows);
  if (e != cudaSuccess || !addr) {
    *why = e;
    return 2;
  }
  double* rows = static_cast<double*>(addr);
  cudaMemsetAsync(dst, 0, sizeof(double) * (size_t)(g.nx + 1) * (g.nz + 1), s);
  if (cap > 0) {
    k_rho<T><<<(cap + 255) / 256, 256, 0, s>>>(g, p, ctrl, order, -kQe, dst);
    (*kernels)++;
  }
  if (ions) {
    // the same row-density kernel as the step, at one time (both outputs alias the scratch)
    k_ion_rows<<<dim3((g.nz + 1 + 7) / 8, 1), 256, 0, s>>>(g, mlo, mhi, t, t, ip, order, rows, rows);
    launch_ion_rho(g, ion_x, rows, kQe / (g.dx * g.dz), dst, s);
    *kernels += 2;
  }
  const cudaError_t le = cudaGetLastError();
  if (le != cudaSuccess) {
    *why = le;
    return 3;
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Self-field of the frozen test beam (Sec. 3.1.1: the fields at the injection plane must be consistent with
// the beam). The frozen charge moves rigidly at the beam's mean velocity v along z, so in the computational
// frame the potential solves d2phi/dx2 + d2phi/dz2 / gamma_v^2 = -rho/eps0 with phi = 0 on the grid edges
// (the PEC walls), discretised with the Yee mesh's second differences; E_x = -dphi/dx, E_z = -dphi/dz /
// gamma_v^2 at their half positions and B_y = v E_x / c^2 (PR-27). The sine transform (DST-I) diagonalises
// the discrete operator: phi_hat(m, q) = -rho_hat(m, q) / (eps0 (lx(m) + lz(q) / gamma_v^2)) with
// lx(m) = -(2 - 2 cos(pi m / nx)) / dx^2, lz likewise. The transforms are direct sums over a sine table,
// FP64 throughout (a one-time set-up: O(nx nz (nx + nz)) multiply-adds).

// charge density (nx+1) x (nz+1) of the frozen beam particles inside the particle domain, their positions
// taken `shift` seconds from now (frozen particles move at v)
template <class T>
__global__ void k_beam_rho(GridP g, Beam<T> b, int order, double shift, const double* acc, double* rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  if ((b.flag[j] & 3) != 1) return;   // alive and frozen only
  const double v = acc[2];
  const double x = b.x[j], z = b.z[j] + v * shift;
  const double xlo = g.gx_lo * g.dx, xhi = g.gx_hi * g.dx;
  const double zlo = g.z0 + g.gz_lo * g.dz, zhi = g.z0 + (g.gz_hi + 1) * g.dz;
  if (!(x >= xlo && x < xhi && z >= zlo && z < zhi)) return;
  const double qw = -kQe * (double)b.w[j];
  const double X = x / g.dx, Z = (z - g.z0) / g.dz;
  const int fx = (int)floor(X), fz = (int)floor(Z);
  for (int i = fx - 2; i <= fx + 3; i++)
    for (int k = fz - 2; k <= fz + 3; k++) {
      const double sv = shape_val(order, X - i) * shape_val(order, Z - k);
      if (sv != 0.0 && i >= 0 && i <= g.nx && k >= 0 && k <= g.nz)
        atomicAdd(&rho[(long)i * (g.nz + 1) + k], qw * sv / (g.dx * g.dz));
    }
}

// out(o, m) = 2 sum_{j=1}^{N-1} in(o, j) sin(pi j m / N) for m = 1..N-1 and rows o = 1..n_outer-1, the
// transform index running with stride si, the rows with stride so; tab[t] = sin(pi t / N), t < 2N. One
// thread per (o, m); the table index j m mod 2N advances by m per term.
__global__ void k_dst1(const double* in, double* out, const double* tab, int N, int n_outer, long so, long si) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long n_m = N - 1, n_o = n_outer - 1;
  if (id >= n_m * n_o) return;
  long o, m;
  if (si == 1) { o = 1 + id / n_m; m = 1 + id % n_m; }     // transform along the fast axis: threads over m
  else { m = 1 + id / n_o; o = 1 + id % n_o; }             // along the slow axis: threads over the rows
  const double* src = in + o * so;
  const int twoN = 2 * N;
  int t = 0;
  double acc = 0.0;
  for (int jj = 1; jj < N; jj++) {
    t += (int)m;
    if (t >= twoN) t -= twoN;
    acc += src[(long)jj * si] * tab[t];
  }
  out[o * so + m * si] = 2.0 * acc;
}

__global__ void k_poisson_divide(double* a, int nx, int nz, double dx, double dz, double gv2) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long)(nx - 1) * (nz - 1)) return;
  const int m = 1 + (int)(id / (nz - 1)), q = 1 + (int)(id % (nz - 1));
  const double lx = -(2.0 - 2.0 * cospi((double)m / nx)) / (dx * dx);
  const double lz = -(2.0 - 2.0 * cospi((double)q / nz)) / (dz * dz);
  // the inverse DST-I of each axis is the forward one over 2N
  const long p = (long)m * (nz + 1) + q;
  a[p] = -a[p] / kEps0 / (lx + lz / gv2) / (4.0 * nx * nz);
}

// E_x, E_z from phi (mode 0) or B_y from phi (mode 1) added to the context's fields
template <class T>
__global__ void k_self_field_add(GridP g, FieldPtrs<T> f, const double* phi, double gv2, const double* acc, int mode) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (k > g.nz) return;
  const int L = g.nz + 1;
  const long q = (long)i * g.ld + k;
  const double* P = phi + (long)i * L;
  if (mode == 0) {
    if (i < g.nx) f.E[0][q] += T(-(P[L + k] - P[k]) / g.dx);
    if (k < g.nz) f.E[2][q] += T(-(P[k + 1] - P[k]) / g.dz / gv2);
  } else if (i < g.nx && k < g.nz) {
    const double ex0 = -(P[L + k] - P[k]) / g.dx, ex1 = -(P[L + k + 1] - P[k + 1]) / g.dx;
    f.B[1][q] += T(acc[2] / (kC * kC) * 0.5 * (ex0 + ex1));
  }
}

// phi is zero on the grid's edges (the transforms leave the deposited density there)
__global__ void k_zero_edges(double* a, int nx, int nz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = nz + 1;
  if (t <= nz) { a[t] = 0.0; a[(long)nx * L + t] = 0.0; }
  if (t <= nx) { a[(long)t * L] = 0.0; a[(long)t * L + nz] = 0.0; }
}

template <class T>
void launch_beam_self_field(const GridP& g, const FieldPtrs<T>& f, Beam<T> b, int order, const double* acc,
                            double gv2, double* rho, double* tmp, double* tabx, double* tabz, cudaStream_t s) {
  const size_t n = (size_t)(g.nx + 1) * (g.nz + 1);
  const int L = g.nz + 1;
  for (int mode = 0; mode < 2; mode++) {
    // E from the positions now, B_y half a step earlier (B^{n-1/2})
    cudaMemsetAsync(rho, 0, n * sizeof(double), s);
    cudaMemsetAsync(tmp, 0, n * sizeof(double), s);
    if (b.n > 0) k_beam_rho<T><<<(b.n + 255) / 256, 256, 0, s>>>(g, b, order, mode == 0 ? 0.0 : -0.5 * g.dt, acc, rho);
    const long nz_work = (long)(g.nx - 1) * (g.nz - 1);
    const unsigned blocks = (unsigned)((nz_work + 255) / 256);
    // forward: along z (rows i), then along x (columns k)
    k_dst1<<<blocks, 256, 0, s>>>(rho, tmp, tabz, g.nz, g.nx, L, 1);
    k_dst1<<<blocks, 256, 0, s>>>(tmp, rho, tabx, g.nx, g.nz, 1, L);
    k_poisson_divide<<<blocks, 256, 0, s>>>(rho, g.nx, g.nz, g.dx, g.dz, gv2);
    // inverse (the same transforms; the 1/(4 nx nz) is in the division)
    k_dst1<<<blocks, 256, 0, s>>>(rho, tmp, tabz, g.nz, g.nx, L, 1);
    k_dst1<<<blocks, 256, 0, s>>>(tmp, rho, tabx, g.nx, g.nz, 1, L);
    k_zero_edges<<<(max(g.nx, g.nz) + 1 + 255) / 256, 256, 0, s>>>(rho, g.nx, g.nz);
    dim3 grd((g.nz + 1 + 255) / 256, g.nx + 1);
    k_self_field_add<T><<<grd, 256, 0, s>>>(g, f, rho, gv2, acc, mode);
  }
}

void launch_ion_column(const GridP& g, long long mlo, long long mhi, double t0, double t1, const InjectP& ip,
                       int order, double* C, cudaStream_t s) {
  cudaMemsetAsync(C, 0, sizeof(double) * (size_t)(g.nz + 1), s);
  const long long n = mhi - mlo;
  if (n > 0) k_ion_current<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(g, mlo, mhi, t0, t1, ip, order, C);
}

void launch_ion_rows(const GridP& g, long long mlo, long long mhi, double t, const InjectP& ip, int order, double* R,
                     cudaStream_t s) {
  k_ion_rows<<<dim3((g.nz + 1 + 7) / 8, 1), 256, 0, s>>>(g, mlo, mhi, t, t, ip, order, R, R);
}

template <class T>
void launch_antenna(const GridP& g, T* Jy, const double* xs, const AntennaStep& a, cudaStream_t s) {
  k_antenna<T><<<(g.nx + 1 + 127) / 128, 128, 0, s>>>(g, Jy, xs, a);
}

template <class T>
void launch_beam_init(Beam<T> b, const double* lx, const double* lz, const double* lux, const double* luy,
                      const double* luz, double t_lab, double z_plane, double gamma, double beta, double t_now,
                      double* scratch, cudaStream_t s) {
  cudaMemsetAsync(scratch, 0, 4 * sizeof(double), s);
  const int nb = (b.n + 255) / 256;
  k_beam_sum_vz<<<nb, 256, 0, s>>>(b.n, lux, luy, luz, scratch);
  k_beam_transform<T><<<nb, 256, 0, s>>>(b, lx, lz, lux, luy, luz, t_lab, z_plane, gamma, beta, scratch);
  k_beam_finish<T><<<nb, 256, 0, s>>>(b, t_now, scratch);
}

template <class T>
void launch_beam_push_batch(const StepArgs<T>* a, int nruns, int beam_blocks, cudaStream_t s) {
  if (beam_blocks > 0) k_beam_push_batch<T><<<dim3(beam_blocks, nruns), 128, 0, s>>>(a);
}

template <class T>
void launch_beam_push(const GridP& g, const FieldPtrs<T>& f, Beam<T> b, int order, double tn, double tn1, int nodal,
                      const double* scratch, cudaStream_t s) {
  if (b.n <= 0) return;
  k_beam_push<T><<<(b.n + 127) / 128, 128, 0, s>>>(g, f, b, order, tn, tn1, nodal, scratch);
}

// 'momentum conserving' gather (Sec. 5): each gather copy interpolated to the nodes, the mean of its two
// nearest values along each half-integer axis (four for B_y, staggered along x and z); values off the
// grid count as zero
template <class T>
__global__ void k_nodal(GridP g, FieldPtrs<T> f) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (k > g.nz) return;
  const long q = (long)i * g.ld + k;
  const bool il = i >= 1, kl = k >= 1;
  const long qx = q - g.ld, qz = q - 1, qxz = q - g.ld - 1;
  const T* Ex = f.fE[0];
  const T* Ez = f.fE[2];
  const T* Bx = f.fB[0];
  const T* By = f.fB[1];
  const T* Bz = f.fB[2];
  f.nE[0][q] = T(0.5) * ((il ? Ex[qx] : T(0)) + Ex[q]);
  f.nE[1][q] = f.fE[1][q];
  f.nE[2][q] = T(0.5) * ((kl ? Ez[qz] : T(0)) + Ez[q]);
  f.nB[0][q] = T(0.5) * ((kl ? Bx[qz] : T(0)) + Bx[q]);
  f.nB[1][q] = T(0.25) * ((il && kl ? By[qxz] : T(0)) + (kl ? By[qz] : T(0)) + (il ? By[qx] : T(0)) + By[q]);
  f.nB[2][q] = T(0.5) * ((il ? Bz[qx] : T(0)) + Bz[q]);
}

template <class T>
void launch_nodal(const GridP& g, const FieldPtrs<T>& f, cudaStream_t s) {
  k_nodal<T><<<dim3((g.nz + 1 + 127) / 128, g.nx + 1), 128, 0, s>>>(g, f);
}

template <class T>
void launch_btd(const GridP& g, const FieldPtrs<T>& f, int which, int post, int r0, int r1, const int* order_idx,
                const double* tp, const double* zp, double ta, double gamma, double beta, T* out, int* done,
                cudaStream_t s) {
  if (r1 <= r0) return;
  dim3 grd((g.nx + 1 + 127) / 128, r1 - r0);
  k_btd<T><<<grd, 128, 0, s>>>(g, f, which, post, r0, r1, order_idx, tp, zp, ta, gamma, beta, out, done);
}

template <class T>
void launch_rho(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int order, double q, double* rho,
                cudaStream_t s) {
  if (cap <= 0) return;
  k_rho<T><<<(cap + 255) / 256, 256, 0, s>>>(g, p, ctrl, order, q, rho);
}

void launch_ion_rho(const GridP& g, const double* ion_x, const double* R, double coef, double* rho, cudaStream_t s) {
  dim3 grd((g.nz + 1 + 255) / 256, g.nx + 1);
  k_ion_rho<<<grd, 256, 0, s>>>(g, ion_x, R, coef, rho);
}

template <class T>
void launch_stats(const GridP& g, const FieldPtrs<T>& f, Particles<T> p, const Ctrl* ctrl, int cap, Beam<T> b,
                  double gamma, double beta, double trap, double* out, cudaStream_t s) {
  (void)cap;
  cudaMemsetAsync(out, 0, 8 * sizeof(double), s);
  k_stats<T><<<152 * 8, 256, 0, s>>>(g, f, p, ctrl, b, gamma, beta, trap, out);
}

template <class T>
void launch_shift(const GridP& g, T* arr, T* tmp, int sh, int comp, cudaStream_t s) {
  dim3 grd((g.nz + 1 + 255) / 256, g.nx + 1);
  k_shift_copy<T><<<grd, 256, 0, s>>>(g, arr, tmp, sh, comp);
  cudaMemcpyAsync(arr, tmp, sizeof(T) * (size_t)(g.nx + 1) * g.ld, cudaMemcpyDeviceToDevice, s);
}

void launch_shift_chunks(Chunk* chunks, Ctrl* ctrl, int sh, int chunk_cap, cudaStream_t s) {
  k_shift_chunks<<<(chunk_cap + 255) / 256, 256, 0, s>>>(chunks, ctrl, sh);
}

template <class T>
void launch_convert(const T* src, double* dst, const GridP& g, cudaStream_t s) {
  dim3 grd((g.nz + 1 + 255) / 256, g.nx + 1);
  k_convert<T><<<grd, 256, 0, s>>>(src, dst, g);
}

template <class T>
void launch_convert_back(const double* src, T* dst, const GridP& g, cudaStream_t s) {
  dim3 grd((g.nz + 1 + 255) / 256, g.nx + 1);
  k_convert_back<T><<<grd, 256, 0, s>>>(src, dst, g);
}

template <class T>
void launch_compact_copy(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, double* out6, uint32_t* id_out,
                         int* nout, cudaStream_t s) {
  cudaMemsetAsync(nout, 0, sizeof(int), s);
  if (cap <= 0) return;
  k_compact<T><<<(cap + 255) / 256, 256, 0, s>>>(g, p, ctrl, out6, id_out, nout, cap);
}

template <class T>
void launch_shift_particles(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int sh, cudaStream_t s) {
  if constexpr (CellPos<T>::value) {
    if (cap > 0) k_shift_particles<T><<<(cap + 255) / 256, 256, 0, s>>>(g, p, ctrl, sh);
  }
}

#define INST(T)                                                                                                   \
  template void launch_antenna<T>(const GridP&, T*, const double*, const AntennaStep&, cudaStream_t);           \
  template void launch_beam_init<T>(Beam<T>, const double*, const double*, const double*, const double*,          \
                                    const double*, double, double, double, double, double, double*, cudaStream_t); \
  template void launch_antenna_ion_batch<T>(const StepArgs<T>*, const BatchGrid&, bool, cudaStream_t);          \
  template void launch_beam_self_field<T>(const GridP&, const FieldPtrs<T>&, Beam<T>, int, const double*, double, \
                                          double*, double*, double*, double*, cudaStream_t);                    \
  template void launch_beam_push_batch<T>(const StepArgs<T>*, int, int, cudaStream_t);                              \
  template void launch_beam_push<T>(const GridP&, const FieldPtrs<T>&, Beam<T>, int, double, double, int,         \
                                    const double*, cudaStream_t);                                                 \
  template void launch_nodal<T>(const GridP&, const FieldPtrs<T>&, cudaStream_t);                                 \
  template void launch_btd<T>(const GridP&, const FieldPtrs<T>&, int, int, int, int, const int*, const double*,   \
                              const double*, double, double, double, T*, int*, cudaStream_t);                     \
  template void launch_rho<T>(const GridP&, Particles<T>, const Ctrl*, int, int, double, double*, cudaStream_t);  \
  template void launch_stats<T>(const GridP&, const FieldPtrs<T>&, Particles<T>, const Ctrl*, int, Beam<T>,       \
                                double, double, double, double*, cudaStream_t);                                           \
  template void launch_shift<T>(const GridP&, T*, T*, int, int, cudaStream_t);                                        \
  template void launch_convert<T>(const T*, double*, const GridP&, cudaStream_t);                                \
  template void launch_convert_back<T>(const double*, T*, const GridP&, cudaStream_t);                           \
  template void launch_compact_copy<T>(const GridP&, Particles<T>, const Ctrl*, int, double*, uint32_t*, int*,      \
                                       cudaStream_t);                                                             \
  template void launch_shift_particles<T>(const GridP&, Particles<T>, const Ctrl*, int, int, cudaStream_t);                 \
  template int launch_rho_noalloc<T>(const GridP&, Particles<T>, const Ctrl*, int, int, bool, long long,         \
                                     long long, double, const InjectP&, const double*, double*, cudaStream_t,   \
                                     cudaError_t*, int*);
INST(float)
INST(double)
#undef INST

}  // namespace picgb
