// 1D path (z only; fields and positions depend on z, the three momentum
// components are kept) of the boosted-frame PIC step (Vay et al.,
// arXiv:1009.2727): the 2D/3D scheme with d/dx = d/dy = 0, which is Eq. 1db-1de
// of App. I for the transverse pair plus E_z from the longitudinal current.
//  - Faraday (the enlarged operator reduces to the Yee difference in 1D) with
//    Friedman's E_eff and the PML at both ends; Ampère with the PML;
//  - the composed filter along z (passes, compensation, stride or a set);
//  - gather (Yee locations or node-interpolated), Boris, 1D Esirkepov deposit;
//  - plasma rows through z_hi, ions fixed in the lab as a column current, a
//    current-sheet antenna, the lab-frame moving window.
// Layout: node k of every component at index k (arrays padded to 32 values);
// Ex, Ey, Bz, Jx, Jy at k, Ez, Bx, By, Jz at k + 1/2. Weights per unit area.
// One thread per node for the fields; one thread per particle for the push,
// whose deposit adds to the current with global atomics (1D grids are small:
// the step is launch-bound, not bandwidth-bound).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pic_3d.h"
#include "pic_common.cuh"

namespace picgb {
namespace {

struct G1 {
  int nz;          // cells
  int n1p;         // padded node count of every array
  int lo, hi;      // particle domain [cells]
  double dz, idz, dt, z0;
};

inline unsigned nb1(long n, int b) { return (unsigned)((n + b - 1) / b); }

// valid range of component c (0..5: E then B; 6..8: J like E): half-staggered 0..nz-1, integer E 1..nz-1
// (tangential E vanishes on the PEC walls), integer B (Bz) 0..nz
__host__ __device__ inline bool half1(int c) {
  const int q = c >= 6 ? c - 6 : c;
  return q == 2 || q == 3 || q == 4;
}
__host__ __device__ inline void vr1(int c, int nz, int& lo, int& hi) {
  const int q = c >= 6 ? c - 6 : c;
  if (half1(q)) { lo = 0; hi = nz - 1; }
  else if (q < 3) { lo = 1; hi = nz - 1; }
  else { lo = 0; hi = nz; }
}

// B-spline shape of order 1 or 3 at offset s (cells)
template <class R>
__device__ __forceinline__ R shp(int order, R s) {
  const R a = fabs(s);
  if (order == 1) return a < R(1) ? R(1) - a : R(0);
  if (a < R(1)) return R(2) / R(3) - a * a + R(0.5) * a * a * a;
  if (a < R(2)) { const R t = R(2) - a; return t * t * t / R(6); }
  return R(0);
}

template <class T>
struct Pml1 {
  const T *sgI, *xiI, *cfI;   // integer positions
  const T *sgH, *xiH, *cfH;   // half positions
};

template <class T>
struct Taps1 {
  T c[2 * FILTER_HMAX + 1];
  int P, s;
};

// ---------------------------------------------------------------------------
// fields
// moving window: every field array moves down by sh cells, keeping each component on its valid range
template <class T>
__global__ void k1_shift(G1 g, T* const* arr, const int* comp, int sh) {
  const int a = blockIdx.y;
  T* F = arr[a];
  const int c = comp[a];
  int lo, hi;
  vr1(c, g.nz, lo, hi);
  // in-place downward copy by one block per array, chunk by chunk from the bottom: a node reads a higher
  // index than it writes, and every read of a chunk precedes its writes (1D grids are small)
  for (int k0 = 0; k0 <= g.nz; k0 += blockDim.x) {
    const int k = k0 + threadIdx.x;
    T v = T(0);
    if (k <= g.nz) {
      const int kk = k + sh;
      v = kk <= g.nz ? F[kk] : T(0);
    }
    __syncthreads();
    if (k <= g.nz) F[k] = (k >= lo && k <= hi) ? v : T(0);
    __syncthreads();
  }
}

// Faraday with E_eff = c1 E - c2 E^{n-1} + c3 E-bar and the PML: Bx(k+1/2) += dt dEy/dz,
// By(k+1/2) -= dt dEx/dz; Bavg = (B^{n-1/2} + B^{n+1/2}) / 2 for the gather
template <class T>
__global__ void k1_faraday(G1 g, Pml1<T> pm, const T* E, const T* Ep, const T* Eb, T* B, T* Bavg, T c1, T c2, T c3,
                           T dtT, T idz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const int n = g.n1p;
  for (int q = 0; q < 3; q++) {
    const T old = B[q * n + k];
    T nw = old;
    if (q < 2 && k <= g.nz - 1) {
      const int ce = q == 0 ? 1 : 0;
      const T sgn = q == 0 ? T(1) : T(-1);
      const T e1 = c1 * E[ce * n + k + 1] - c2 * Ep[ce * n + k + 1] + c3 * Eb[ce * n + k + 1];
      const T e0 = c1 * E[ce * n + k] - c2 * Ep[ce * n + k] + c3 * Eb[ce * n + k];
      const T d = sgn * (e1 - e0) * idz;
      const T sg = pm.sgH[k];
      nw = sg > T(0) ? pm.xiH[k] * old + pm.cfH[k] * d : old + dtT * d;
      B[q * n + k] = nw;
    }
    Bavg[q * n + k] = T(0.5) * (old + nw);
  }
}

// Friedman history (PR-1): E-bar <- (1 - theta/2) E + (theta/2) E-bar, E^{n-1} <- E
template <class T>
__global__ void k1_friedman(int n, const T* E, T* Ep, T* Eb, T a, T b) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const T e = E[p];
  Eb[p] = a * e + b * Eb[p];
  Ep[p] = e;
}

// composed filter along z on up to six components (blockIdx.y): dst = sum_m c_m src(k + (m - P) s), zero
// off the component's valid range and off the grid
template <class T>
struct FiltJob1 {
  const T* src[6];
  T* dst[6];
  int comp[6];
};

template <class T>
__global__ void k1_filter(G1 g, FiltJob1<T> jb, Taps1<T> t) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const int a = blockIdx.y;
  const T* F = jb.src[a];
  int lo, hi;
  vr1(jb.comp[a], g.nz, lo, hi);
  T acc = T(0);
  if (k >= lo && k <= hi) {
    for (int m = 0; m <= 2 * t.P; m++) {
      const int o = k + (m - t.P) * t.s;
      if (o >= 0 && o <= g.nz) acc += t.c[m] * F[o];
    }
  }
  jb.dst[a][k] = acc;
}

// 'momentum conserving' gather (Sec. 5): node values of the six gather copies, the mean of the two
// nearest values of a half-staggered component (Ez, Bx, By); values off the grid count as zero
template <class T>
__global__ void k1_nodal(G1 g, const T* fE, const T* fB, T* dst) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const int n = g.n1p;
  for (int c = 0; c < 6; c++) {
    const T* F = c < 3 ? fE + c * n : fB + (c - 3) * n;
    dst[c * n + k] = half1(c) ? T(0.5) * ((k >= 1 ? F[k - 1] : T(0)) + F[k]) : F[k];
  }
}

// Ampère with the PML: Ex(k) += dt (-c^2 dBy/dz - Jx/eps0), Ey(k) += dt (c^2 dBx/dz - Jy/eps0),
// Ez(k+1/2) += -dt Jz/eps0; no current in the PML, where the curl term is damped
template <class T>
__global__ void k1_ampere(G1 g, Pml1<T> pm, T* E, const T* B, const T* J, T dtT, T c2idz, T ie0) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const int n = g.n1p;
  for (int q = 0; q < 3; q++) {
    int lo, hi;
    vr1(q, g.nz, lo, hi);
    if (k < lo || k > hi) continue;
    T d = T(0);
    if (q == 0) d = -c2idz * (B[1 * n + k] - (k >= 1 ? B[1 * n + k - 1] : T(0)));
    if (q == 1) d = c2idz * (B[0 * n + k] - (k >= 1 ? B[0 * n + k - 1] : T(0)));
    const T sg = q == 2 ? pm.sgH[k] : pm.sgI[k];
    T& e = E[q * n + k];
    if (sg > T(0)) e = (q == 2 ? pm.xiH[k] : pm.xiI[k]) * e + (q == 2 ? pm.cfH[k] : pm.cfI[k]) * d;
    else e = e + dtT * (d - J[q * n + k] * ie0);
  }
}

// ---------------------------------------------------------------------------
// particles
template <class T>
struct Parts1 {
  double* z;
  T *ux, *uy, *uz, *w;
  uint32_t* id;
};

struct Ctrl1 {
  int count;
  int status;
};

// one electron per thread: gather -> Boris -> move -> 1D Esirkepov; removal after the deposit when it
// leaves [z_lo, z_hi + dz). The particles of a block are consecutive in memory and, injected row by row,
// close in z: their current is summed in a shared window over the block's cells (one global atomic per
// window node afterwards), else, for a block spread wider than the window, added to J directly.
constexpr int PB1 = 128, JW1 = 320;
template <class T, bool MC>
__global__ void __launch_bounds__(PB1) k1_push(G1 g, const T* fE, const T* fB, T* J, Parts1<T> p, const Ctrl1* ctrl,
                                               int order, T kq, T qe, double zlo, double zhi1) {
  __shared__ T sJ[3][JW1];
  __shared__ int s_lo, s_hi;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = g.n1p;
  if (threadIdx.x == 0) { s_lo = INT_MAX; s_hi = INT_MIN; }
  for (int e = threadIdx.x; e < 3 * JW1; e += blockDim.x) (&sJ[0][0])[e] = T(0);
  __syncthreads();
  const bool live = j < ctrl->count && p.w[j] > T(0);
  double z = 0.0, Z = 0.0;
  int f = 0;
  if (live) {
    z = p.z[j];
    Z = (z - g.z0) * g.idz;
    f = (int)floor(Z);
    atomicMin(&s_lo, f);
    atomicMax(&s_hi, f);
  }
  __syncthreads();
  // the deposit of a particle in cell f (moving less than a cell) touches nodes f - 4 .. f + 5
  const int base = s_lo - 5, span = s_hi - s_lo + 12;
  const bool win = s_hi >= s_lo && span <= JW1;
  if (live) {
    const T w = p.w[j];
    T EB[6];
#pragma unroll
    for (int c = 0; c < 6; c++) {
      const T* F = c < 3 ? fE + c * n : fB + (c - 3) * n;
      const double st = (!MC && half1(c)) ? 0.5 : 0.0;
      T acc = T(0);
      for (int k = f - 3; k <= f + 3; k++) {
        if (k < 0 || k > g.nz) continue;
        const T wz = shp<T>(order, T(Z - (k + st)));
        if (wz != T(0)) acc += F[k] * wz;
      }
      EB[c] = acc;
    }
    // relativistic Boris push (textbook)
    T u0 = p.ux[j], u1 = p.uy[j], u2 = p.uz[j];
    const T ic2 = T(1.0 / (kC * kC));
    const T um0 = u0 + kq * EB[0], um1 = u1 + kq * EB[1], um2 = u2 + kq * EB[2];
    const T gm = sqrt(T(1) + (um0 * um0 + um1 * um1 + um2 * um2) * ic2);
    const T t0 = kq * EB[3] / gm, t1 = kq * EB[4] / gm, t2 = kq * EB[5] / gm;
    const T tt = t0 * t0 + t1 * t1 + t2 * t2;
    const T s0 = T(2) * t0 / (T(1) + tt), s1 = T(2) * t1 / (T(1) + tt), s2 = T(2) * t2 / (T(1) + tt);
    const T up0 = um0 + (um1 * t2 - um2 * t1), up1 = um1 + (um2 * t0 - um0 * t2), up2 = um2 + (um0 * t1 - um1 * t0);
    const T pl0 = um0 + (up1 * s2 - up2 * s1), pl1 = um1 + (up2 * s0 - up0 * s2), pl2 = um2 + (up0 * s1 - up1 * s0);
    u0 = pl0 + kq * EB[0]; u1 = pl1 + kq * EB[1]; u2 = pl2 + kq * EB[2];
    const T g1 = sqrt(T(1) + (u0 * u0 + u1 * u1 + u2 * u2) * ic2);
    const double zn = z + g.dt * (double)(u2 / g1);
    const double Zn = (zn - g.z0) * g.idz;
    // 1D Esirkepov: Jz(k+1/2) = -(q w/dt) sum_{k' <= k} (S1 - S0)(k'); Jx, Jy = q w v (S0 + S1)/(2 dz)
    const T qw = qe * w;
    const T vx = u0 / g1, vy = u1 / g1;
    const T cz = -qw / T(g.dt), ct = qw * T(0.5) * T(g.idz);
    const int b = (int)floor(Z < Zn ? Z : Zn) - 3;
    T run = T(0);
    for (int a = 0; a < 9; a++) {
      const int k = b + a;
      const T S0 = shp<T>(order, T(Z - k)), S1 = shp<T>(order, T(Zn - k));
      run += S1 - S0;
      if (k < 0 || k > g.nz) continue;
      const T ss = S0 + S1;
      const T jz = cz * run, jx = ct * vx * ss, jy = ct * vy * ss;
      const int l = k - base;
      if (win && l >= 0 && l < span) {
        if (jz != T(0)) atomicAdd(&sJ[2][l], jz);
        if (jx != T(0)) atomicAdd(&sJ[0][l], jx);
        if (jy != T(0)) atomicAdd(&sJ[1][l], jy);
      } else {
        if (jz != T(0)) atomicAdd(J + 2 * n + k, jz);
        if (jx != T(0)) atomicAdd(J + k, jx);
        if (jy != T(0)) atomicAdd(J + n + k, jy);
      }
    }
    p.z[j] = zn;
    p.ux[j] = u0; p.uy[j] = u1; p.uz[j] = u2;
    if (zn < zlo || zn >= zhi1) p.w[j] = T(0);
  }
  __syncthreads();
  if (win) {
    for (int e = threadIdx.x; e < 3 * span; e += blockDim.x) {
      const int q = e / span, l = e - q * span, k = base + l;
      const T v = sJ[q][l];
      if (v != T(0) && k >= 0 && k <= g.nz) atomicAdd(J + q * n + k, v);
    }
  }
}

// plasma rows [m0, m0 + nrow): row m at z' = (m + 1/2) h - beta c t, density gamma n0(gamma (m + 1/2) h),
// weight n' dz / ppc_z per unit area; rows without plasma, or below z_lo, are stored dead (w = 0)
struct Lat1 {
  double h, gamma, beta, n0, z_start_lab, ramp_lab, length_lab, dz;
  int ppc;
};

__host__ __device__ inline double lab_density1(const Lat1& L, double zl) {
  if (zl < L.z_start_lab) return 0.0;
  const double r = zl - L.z_start_lab;
  if (L.ramp_lab > 0.0 && r < L.ramp_lab) return L.n0 * r / L.ramp_lab;
  const double plateau_end = L.ramp_lab + L.length_lab;
  if (L.length_lab > 0.0 && r >= plateau_end) return 0.0;
  return L.n0;
}

template <class T>
__global__ void k1_inject(Parts1<T> p, Ctrl1* ctrl, Lat1 L, long long m0, int nrow, double t, double zlo, int at) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrow) return;
  const long long m = m0 + r;
  const double zlat = (m + 0.5) * L.h;
  const double n = L.gamma * lab_density1(L, L.gamma * zlat);
  const double zp = zlat - L.beta * kC * t;
  const int q = at + r;
  p.z[q] = zp;
  p.ux[q] = T(0);
  p.uy[q] = T(0);
  p.uz[q] = T(-L.gamma * L.beta * kC);
  p.w[q] = (n > 0.0 && zp >= zlo) ? T(n * L.dz / (double)L.ppc) : T(0);
  p.id[q] = (uint32_t)m;
  if (r == 0) ctrl->count = at + nrow;
}

// sum over n >= 0 of S(u + n): the prefix of the shape samples (the 1D Esirkepov flux of a row)
__device__ __forceinline__ double cum_shape1(int order, double u) {
  const double r = order == 3 ? 2.0 : 1.0;
  if (u >= r) return 0.0;
  if (u <= -r) return 1.0;
  double acc = 0.0;
  for (int n = 0; n < 5; n++) acc += shp<double>(order, u + n);
  return acc;
}

// ions fixed in the lab (PR-9): J_z(k+1/2) += -(e/dt) sum over the live rows of w_m (C(Z1 - k) - C(Z0 - k))
template <class T>
__global__ void k1_ion_jz(G1 g, Lat1 L, int order, long long mlo, long long mhi, double t0, double t1, T* Jz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const double vsh = L.beta * kC;
  long long m0 = (long long)floor(((k - 4) * g.dz + g.z0 + vsh * t0) / L.h - 0.5);
  long long m1 = (long long)ceil(((k + 4) * g.dz + g.z0 + vsh * t0) / L.h - 0.5);
  if (m0 < mlo) m0 = mlo;
  if (m1 > mhi - 1) m1 = mhi - 1;
  double acc = 0.0;
  for (long long m = m0; m <= m1; m++) {
    const double zl = (m + 0.5) * L.h;
    const double n = L.gamma * lab_density1(L, L.gamma * zl);
    if (n <= 0.0) continue;
    const double w = n * L.dz / (double)L.ppc;
    const double Z0 = (zl - vsh * t0 - g.z0) * g.idz, Z1 = (zl - vsh * t1 - g.z0) * g.idz;
    acc += w * (cum_shape1(order, Z1 - k) - cum_shape1(order, Z0 - k));
  }
  if (acc != 0.0) Jz[k] += T(-kQe / g.dt * acc);
}

// charge density: electrons and the ion rows at time t
template <class T>
__global__ void k1_rho_e(G1 g, Parts1<T> p, const Ctrl1* ctrl, int order, double* rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->count) return;
  const double w = (double)p.w[j];
  if (!(w > 0.0)) return;
  const double Z = (p.z[j] - g.z0) * g.idz;
  const int f = (int)floor(Z);
  for (int k = f - 3; k <= f + 3; k++) {
    if (k < 0 || k > g.nz) continue;
    const double s = shp<double>(order, Z - k);
    if (s != 0.0) atomicAdd(rho + k, -kQe * w * s * g.idz);
  }
}

__global__ void k1_rho_i(G1 g, Lat1 L, int order, long long mlo, long long mhi, double t, double* rho) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > g.nz) return;
  const double vsh = L.beta * kC;
  long long m0 = (long long)floor(((k - 3) * g.dz + g.z0 + vsh * t) / L.h - 0.5);
  long long m1 = (long long)ceil(((k + 3) * g.dz + g.z0 + vsh * t) / L.h - 0.5);
  if (m0 < mlo) m0 = mlo;
  if (m1 > mhi - 1) m1 = mhi - 1;
  double acc = 0.0;
  for (long long m = m0; m <= m1; m++) {
    const double zl = (m + 0.5) * L.h;
    const double n = L.gamma * lab_density1(L, L.gamma * zl);
    if (n <= 0.0) continue;
    acc += n * L.dz / (double)L.ppc * shp<double>(order, (zl - vsh * t - g.z0) * g.idz - k);
  }
  rho[k] += kQe * acc * g.idz;
}

// current-sheet antenna: J_y(k) += K w_k / dz over eight nodes from k0
struct Ant1 {
  int k0;
  double v[8];
};
template <class T>
__global__ void k1_antenna(G1 g, Ant1 a, T* Jy) {
  const int i = threadIdx.x;
  const int k = a.k0 + i;
  if (i < 8 && k >= 0 && k <= g.nz && a.v[i] != 0.0) Jy[k] += T(a.v[i]);
}

// diagnostics: [0] live electrons, [1] field energy per unit area, [2] weight above the lab gamma threshold
template <class T>
__global__ void __launch_bounds__(256) k1_stats(G1 g, const T* E, const T* B, Parts1<T> p, const Ctrl1* ctrl,
                                                double gam, double be, double trap, double* out) {
  __shared__ double red[3][256];
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nthr = gridDim.x * blockDim.x;
  double ne = 0, en = 0, wt = 0;
  for (int j = tid; j < ctrl->count; j += nthr) {
    const double w = (double)p.w[j];
    if (!(w > 0.0)) continue;
    ne += 1.0;
    if (trap > 0.0) {
      const double ux = p.ux[j], uy = p.uy[j], uz = p.uz[j];
      const double gp = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
      if (gam * (gp + be * uz / kC) > trap) wt += w;
    }
  }
  const int n = g.n1p;
  for (int k = tid; k <= g.nz; k += nthr) {
    double e2 = 0, b2 = 0;
    for (int c = 0; c < 3; c++) {
      const double ev = E[c * n + k], bv = B[c * n + k];
      e2 += ev * ev; b2 += bv * bv;
    }
    en += 0.5 * (kEps0 * e2 + b2 * (kEps0 * kC * kC)) * g.dz;
  }
  red[0][threadIdx.x] = ne; red[1][threadIdx.x] = en; red[2][threadIdx.x] = wt;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 3; c++) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; c++) atomicAdd(out + c, red[c][0]);
}

// compaction of the live electrons into the other buffer set (order kept)
template <class T>
__global__ void k1_live_per_block(Parts1<T> p, const Ctrl1* ctrl, int* bc) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int live = (j < ctrl->count && p.w[j] > T(0)) ? 1 : 0;
  const int wsum = __popc(__ballot_sync(0xffffffffu, live));
  if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&s, wsum);
  __syncthreads();
  if (threadIdx.x == 0) bc[blockIdx.x] = s;
}

__global__ void __launch_bounds__(1024) k1_scan_blocks(int* bc, int nb, Ctrl1* ctrl) {
  __shared__ int part[1024];
  const int per = (nb + 1023) / 1024;
  const int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
  int s = 0;
  for (int b = b0; b < b1; b++) s += bc[b];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
    __syncthreads();
    part[threadIdx.x] += v;
    __syncthreads();
  }
  int run = part[threadIdx.x] - s;
  for (int b = b0; b < b1; b++) {
    const int c = bc[b];
    bc[b] = run;
    run += c;
  }
  if (threadIdx.x == 1023) ctrl->count = part[1023];
}

template <class T>
__global__ void k1_scatter(Parts1<T> src, Parts1<T> dst, const int* bo, int n_old) {
  __shared__ int wo[8];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int live = (j < n_old && src.w[j] > T(0)) ? 1 : 0;
  const unsigned m = __ballot_sync(0xffffffffu, live);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wo[wid] = __popc(m);
  __syncthreads();
  if (!live) return;
  int off = bo[blockIdx.x];
  for (int q = 0; q < wid; q++) off += wo[q];
  const int d = off + __popc(m & ((1u << lane) - 1u));
  dst.z[d] = src.z[j]; dst.ux[d] = src.ux[j]; dst.uy[d] = src.uy[j]; dst.uz[d] = src.uz[j];
  dst.w[d] = src.w[j]; dst.id[d] = src.id[j];
}

template <class T>
__global__ void k1_out(int n, const T* F, double* out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) out[k] = (double)F[k];
}
template <class T>
__global__ void k1_in(int n, const double* in, T* F) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) F[k] = T(in[k]);
}

// ---------------------------------------------------------------------------
template <class T>
class Sim1 : public Sim3Api {
 public:
  Sim1(const pic_config& c, pic_alloc_fn a, pic_free_fn f, void* u, cudaStream_t s_)
      : cfg(c), alloc(a), freef(f), user(u), s(s_) {}
  ~Sim1() override {
    cudaStreamSynchronize(s);
    for (auto& p : allocs) {
      if (freef) freef(p.first, p.second, (void*)s, user);
      else cudaFree(p.first);
    }
    for (auto e : tev) cudaEventDestroy(e);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }

  int fail(int code, const char* msg) {
    if (st == PIC_OK) { st = code; err = msg; }
    return code;
  }

  template <class U>
  U* dal(size_t n) {
    size_t bytes = std::max<size_t>(n * sizeof(U), 16);
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (alloc) p = alloc(bytes, (void*)s, user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) return nullptr;
    allocs.push_back({p, bytes});
    cudaMemsetAsync(p, 0, bytes, s);
    return (U*)p;
  }

  int init() {
    const pic_config* c = &cfg;
    if (c->nz < 16 || !(c->dz_lab > 0)) return fail(PIC_EINVAL, "1D: nz >= 16 and dz_lab > 0");
    gamma = c->gamma_boost < 1.0 ? 1.0 : c->gamma_boost;
    beta = std::sqrt(1.0 - 1.0 / (gamma * gamma));
    g.nz = c->nz;
    g.n1p = ((c->nz + 1 + 31) / 32) * 32;
    g.dz = (1.0 + beta) * gamma * c->dz_lab;          // Sec. 5.1.1
    g.idz = 1.0 / g.dz;
    g.z0 = 0.0;
    const double th = c->theta;
    const double lim = g.dz / kC * std::sqrt((2.0 + th) / (2.0 + 3.0 * th));
    g.dt = c->dt > 0.0 ? c->dt : c->courant * lim;
    if (!(g.dt > 0.0)) return fail(PIC_EINVAL, "dt <= 0");
    if (g.dt > lim * (1.0 + 1e-12)) return fail(PIC_ECFL, "dt above the 1D stability limit");
    if (c->moving_window && gamma > 1.0) return fail(PIC_EINVAL, "1D moving window: lab frame only");
    FilterSpec fs{};
    fs.passes = c->filter_passes; fs.stride = c->filter_stride; fs.compensate = c->filter_compensate;
    for (int q = 0; q < 4; q++) fs.strides[q] = c->filter_stride_set[q];
    const int H = filter_halo(fs);
    P = c->filter_passes + (c->filter_compensate ? 1 : 0);
    const int guard = c->particle_guard >= 0 ? c->particle_guard : (c->shape_order == 3 ? 3 : 2) + H + 2;
    if (guard < (c->shape_order == 3 ? 3 : 2) + H + 1) return fail(PIC_EINVAL, "particle guard too small");
    g.lo = c->pml_cells + guard;
    g.hi = c->nz - c->pml_cells - guard;
    if (g.hi - g.lo < 2 || g.lo < 4) return fail(PIC_EINVAL, "1D box too small for the PML and guard");
    // composed taps (dense over the halo for a wide-band filter)
    const bool wide = fs.strides[0] > 0;
    const int R = wide ? H : P;
    std::vector<double> t(2 * R + 1, 0.0);
    t[R] = 1.0;
    for (int q = 0; q < (wide ? 4 : 1); q++) {
      const int stq = wide ? fs.strides[q] : 1;
      if (stq <= 0) break;
      for (int pp = 0; pp < P; pp++) {
        const double al = pp < c->filter_passes ? 0.5 : 0.5 * c->filter_passes + 1.0;
        std::vector<double> o(2 * R + 1, 0.0);
        for (int m = 0; m <= 2 * R; m++) {
          o[m] += al * t[m];
          if (m - stq >= 0) o[m] += 0.5 * (1.0 - al) * t[m - stq];
          if (m + stq <= 2 * R) o[m] += 0.5 * (1.0 - al) * t[m + stq];
        }
        t = o;
      }
    }
    for (int m = 0; m < 2 * FILTER_HMAX + 1; m++) taps.c[m] = m <= 2 * R ? T(t[m]) : T(0);
    taps.P = R;
    taps.s = wide ? 1 : c->filter_stride;
    nodal = c->gather_scheme == 1;
    const int n = g.n1p;
    E = dal<T>(3 * n); B = dal<T>(3 * n); J = dal<T>(3 * n); Jf = dal<T>(3 * n); Ep = dal<T>(3 * n);
    Eb = dal<T>(3 * n); Bavg = dal<T>(3 * n); fE = dal<T>(3 * n); fB = dal<T>(3 * n); nF = dal<T>(6 * n);
    rho = dal<double>(n); outd = dal<double>(n); sred = dal<double>(4); ctrl = dal<Ctrl1>(1);
    if (!E || !B || !J || !Jf || !Ep || !Eb || !Bavg || !fE || !fB || !nF || !rho || !outd || !sred || !ctrl)
      return fail(PIC_ENOMEM, "allocation failed");
    // PML tables at integer and half positions
    std::vector<T> sg(2 * n, T(0)), xi(2 * n, T(1)), cf(2 * n, T(g.dt));
    for (int h = 0; h < 2; h++)
      for (int k = 0; k <= c->nz; k++) {
        const double pos = k + 0.5 * h;
        double sgv = 0.0;
        const int L = c->pml_cells;
        if (L > 0) {
          double d = 0.0;
          if (pos < L) d = L - pos;
          if (pos > c->nz - L) d = pos - (c->nz - L);
          if (d > 0.0) sgv = c->pml_sigma_max * kC / g.dz * std::pow(d / c->pml_delta, c->pml_power);
        }
        const double x = c->pml_xi_exp ? std::exp(-sgv * g.dt) : (1.0 - 0.5 * sgv * g.dt) / (1.0 + 0.5 * sgv * g.dt);
        sg[h * n + k] = T(sgv);
        xi[h * n + k] = T(x);
        cf[h * n + k] = T(sgv > 0.0 ? (1.0 - x) / sgv : g.dt);
      }
    T* dsg = dal<T>(2 * n);
    T* dxi = dal<T>(2 * n);
    T* dcf = dal<T>(2 * n);
    if (!dsg || !dxi || !dcf) return fail(PIC_ENOMEM, "allocation failed");
    cudaMemcpyAsync(dsg, sg.data(), sizeof(T) * 2 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dxi, xi.data(), sizeof(T) * 2 * n, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(dcf, cf.data(), sizeof(T) * 2 * n, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    pm.sgI = dsg; pm.xiI = dxi; pm.cfI = dcf;
    pm.sgH = dsg + n; pm.xiH = dxi + n; pm.cfH = dcf + n;
    shift_arr = dal<T*>(12);
    shift_comp = dal<int>(12);
    if (!shift_arr || !shift_comp) return fail(PIC_ENOMEM, "allocation failed");
    T* arrs[12];
    int comps[12];
    for (int q = 0; q < 3; q++) {
      arrs[q] = E + q * n; comps[q] = q;
      arrs[3 + q] = B + q * n; comps[3 + q] = 3 + q;
      arrs[6 + q] = Ep + q * n; comps[6 + q] = q;
      arrs[9 + q] = Eb + q * n; comps[9 + q] = q;
    }
    cudaMemcpyAsync(shift_arr, arrs, sizeof(arrs), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(shift_comp, comps, sizeof(comps), cudaMemcpyHostToDevice, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in 1D init");
  }

  double time_of(long long n) const { return (double)n * g.dt; }
  double z_lo() const { return g.z0 + g.lo * g.dz; }
  double z_hi() const { return g.z0 + g.hi * g.dz; }
  long long rows_inside(double t) const { return (long long)std::ceil((z_hi() + beta * kC * t) / lat.h - 0.5); }

  int alloc_parts(long n) {
    for (int b = 0; b < 2; b++) {
      Parts1<T>& q = P2[b];
      q.z = dal<double>(n); q.ux = dal<T>(n); q.uy = dal<T>(n); q.uz = dal<T>(n); q.w = dal<T>(n);
      q.id = dal<uint32_t>(n);
      if (!q.z || !q.ux || !q.uy || !q.uz || !q.w || !q.id) return PIC_ENOMEM;
    }
    blk = dal<int>(n / 256 + 2);
    if (!blk) return PIC_ENOMEM;
    cap = n;
    return PIC_OK;
  }

  int grow(long need) {
    const long ncap = std::max(need + need / 2, 2 * cap);
    const Parts1<T> o = P2[cur];
    Parts1<T> keep = o;
    if (alloc_parts(ncap) != PIC_OK) return fail(PIC_ENOMEM, "particle allocation failed");
    if (count_ub > 0) {
      const Parts1<T>& d = P2[cur];
      cudaMemcpyAsync(d.z, keep.z, 8 * (size_t)count_ub, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.ux, keep.ux, sizeof(T) * count_ub, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.uy, keep.uy, sizeof(T) * count_ub, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.uz, keep.uz, sizeof(T) * count_ub, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.w, keep.w, sizeof(T) * count_ub, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.id, keep.id, 4 * (size_t)count_ub, cudaMemcpyDeviceToDevice, s);
    }
    return PIC_OK;
  }

  int read_count() {
    Ctrl1 h{};
    cudaMemcpyAsync(&h, ctrl, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return h.count;
  }

  int compact() {
    const int n_old = (int)count_ub;
    if (n_old <= 0) return PIC_OK;
    const int nb = (int)nb1(n_old, 256);
    k1_live_per_block<T><<<nb, 256, 0, s>>>(P2[cur], ctrl, blk);
    k1_scan_blocks<<<1, 1024, 0, s>>>(blk, nb, ctrl);
    k1_scatter<T><<<nb, 256, 0, s>>>(P2[cur], P2[1 - cur], blk, n_old);
    nl += 3;
    cur = 1 - cur;
    const int c = read_count();
    if (c < 0) return fail(PIC_ECUDA, "CUDA error in compaction");
    count_ub = c;
    live_est = c;
    compactions++;
    return PIC_OK;
  }

  int inject(long long m0, long long m1, double t) {
    if (m1 <= m0) return PIC_OK;
    const long nrow = (long)(m1 - m0);
    if (count_ub + nrow > cap && grow(count_ub + nrow) != PIC_OK) return st;
    k1_inject<T><<<nb1(nrow, 128), 128, 0, s>>>(P2[cur], ctrl, lat, m0, (int)nrow, t, z_lo(), (int)count_ub);
    nl++;
    count_ub += nrow;
    live_est += nrow;
    return PIC_OK;
  }

  int load_plasma(const pic_plasma* p) override {
    if (st != PIC_OK) return st;
    if (loaded) return fail(PIC_ESTATE, "plasma already loaded");
    if (p->ppc_z < 1 || p->n0 < 0) return fail(PIC_EINVAL, "bad plasma");
    if (p->beam_n > 0) return fail(PIC_EINVAL, "1D: no test beam");
    lat.h = g.dz / p->ppc_z;
    lat.gamma = gamma; lat.beta = beta;
    lat.n0 = p->n0; lat.z_start_lab = p->z_start_lab; lat.ramp_lab = p->ramp_lab; lat.length_lab = p->length_lab;
    lat.dz = g.dz; lat.ppc = p->ppc_z;
    ions = p->ions != 0;
    const double t = time_of(step);
    const long long m_end = rows_inside(t);
    const long long m_beg = (long long)std::ceil((z_lo() + beta * kC * t) / lat.h - 0.5);
    const long want = (long)(m_end - m_beg) * 2 + 4096;
    if (alloc_parts(want) != PIC_OK) return fail(PIC_ENOMEM, "particle allocation failed");
    count_ub = 0;
    if (inject(m_beg, m_end, t) != PIC_OK) return st;
    row_next = m_end;
    mlo = m_beg;
    loaded = true;
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in plasma load");
  }

  int set_laser(const pic_laser* l) override {
    if (st != PIC_OK) return st;
    if (!(l->lambda0 > 0) || !(l->tau_fwhm > 0)) return fail(PIC_EINVAL, "bad laser");
    if (l->beta_s != 0.0) return fail(PIC_EINVAL, "1D antenna: the plane is at rest in the computational frame");
    las = *l;
    has_laser = true;
    return PIC_OK;
  }

  // the lab waveform E0 exp(-(s - t_peak)^2/(2 sigma^2)) sin(omega (s - t_peak) + phase) emitted from a plane
  // at rest: amplitude and time scaled by (1 + beta) gamma (Sec. 3.1.2, PR-14)
  double emit(double tp) const {
    const double om = 2.0 * kPi * kC / las.lambda0;
    const double E0 = las.a0 * kMe * kC * om / kQe;
    const double dop = (1.0 + beta) * gamma;
    const double sl = tp / dop;
    const double sig = las.tau_fwhm / (2.0 * std::sqrt(std::log(2.0)));
    const double u = sl - las.t_peak;
    return E0 * std::exp(-u * u / (2.0 * sig * sig)) * std::sin(om * u + las.phase) / dop;
  }

  static double shape_h(int order, double s) {
    const double a = std::fabs(s);
    if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
    if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
    if (a < 2.0) { const double t = 2.0 - a; return t * t * t / 6.0; }
    return 0.0;
  }

  // event pairs around the timed launches, read when the timing is queried (no wait inside the step)
  void tbeg(int which) {
    if (!(timing_on && timing_which == which)) return;
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    tev.push_back(a);
    tev.push_back(b);
  }
  void tend(int which) {
    if (!(timing_on && timing_which == which) || tev.empty()) return;
    cudaEventRecord(tev.back(), s);
    t_n++;
  }
  void tcollect() {
    if (tev.empty()) return;
    cudaEventSynchronize(tev.back());
    for (size_t i = 0; i + 1 < tev.size(); i += 2) {
      float ms = 0;
      cudaEventElapsedTime(&ms, tev[i], tev[i + 1]);
      t_ms += ms;
    }
    for (auto e : tev) cudaEventDestroy(e);
    tev.clear();
  }

  int one_step() {
    const int n = g.n1p, n1 = g.nz + 1;
    const double th = cfg.theta;
    const double tn = time_of(step), tn1 = time_of(step + 1);
    // moving window (lab frame): the grid moves down by whole cells
    if (cfg.moving_window) {
      const long long want = (long long)std::floor(cfg.window_beta * kC * tn / g.dz);
      const long long sh = want - shifts;
      if (sh > 0) {
        k1_shift<T><<<dim3(1, 12), 1024, 0, s>>>(g, shift_arr, shift_comp, (int)std::min<long long>(sh, g.nz + 1));
        nl++;
        shifts = want;
        g.z0 = want * g.dz;
      }
    }
    tbeg(1);
    // 1. Faraday + Friedman + PML-B, B average
    k1_faraday<T><<<nb1(n1, 256), 256, 0, s>>>(g, pm, E, Ep, Eb, B, Bavg, T(1.0 + th / 4.0), T(0.5),
                                               T(0.5 - th / 4.0), T(g.dt), T(g.idz));
    k1_friedman<T><<<nb1(3 * n, 256), 256, 0, s>>>(3 * n, E, Ep, Eb, T(1.0 - th / 2.0), T(th / 2.0));
    nl += 2;
    // 2. gather copies (filtered; node-interpolated for the 'momentum conserving' gather)
    const T* gE = E;
    const T* gB = Bavg;
    if (cfg.filter_gather && P > 0) {
      FiltJob1<T> jb;
      for (int q = 0; q < 3; q++) {
        jb.src[q] = E + q * n; jb.dst[q] = fE + q * n; jb.comp[q] = q;
        jb.src[3 + q] = Bavg + q * n; jb.dst[3 + q] = fB + q * n; jb.comp[3 + q] = 3 + q;
      }
      k1_filter<T><<<dim3(nb1(n1, 256), 6), 256, 0, s>>>(g, jb, taps);
      nl++;
      gE = fE; gB = fB;
    }
    if (nodal) {
      k1_nodal<T><<<nb1(n1, 256), 256, 0, s>>>(g, gE, gB, nF);
      nl++;
      gE = nF; gB = nF + 3 * n;
    }
    tend(1);
    // 3. particles
    cudaMemsetAsync(J, 0, sizeof(T) * 3 * n, s);
    tbeg(0);
    if (loaded && count_ub > 0) {
      const T kq = T(-kQe * g.dt / (2.0 * kMe));
      if (nodal)
        k1_push<T, true><<<nb1(count_ub, PB1), PB1, 0, s>>>(g, gE, gB, J, P2[cur], ctrl, cfg.shape_order, kq,
                                                           T(-kQe), z_lo(), z_hi() + g.dz);
      else
        k1_push<T, false><<<nb1(count_ub, PB1), PB1, 0, s>>>(g, gE, gB, J, P2[cur], ctrl, cfg.shape_order, kq,
                                                            T(-kQe), z_lo(), z_hi() + g.dz);
      nl++;
    }
    tend(0);
    // ions fixed in the lab: no current in the lab frame (beta = 0); 32-thread blocks spread the rows' FP64
    // sums over more SMs
    if (loaded && ions && row_next > mlo && beta > 0.0) {
      k1_ion_jz<T><<<nb1(n1, 32), 32, 0, s>>>(g, lat, cfg.shape_order, mlo, row_next, tn, tn1, J + 2 * n);
      nl++;
    }
    // 4. antenna
    if (has_laser && las.z_antenna >= z_lo() && las.z_antenna < z_hi()) {
      const double Z = (las.z_antenna - g.z0) / g.dz;
      const int f = (int)std::floor(Z);
      const double K = -2.0 * kEps0 * kC * emit(0.5 * (tn + tn1));
      Ant1 a;
      a.k0 = f - 3;
      for (int i = 0; i < 8; i++) a.v[i] = K * shape_h(cfg.shape_order, Z - (a.k0 + i)) / g.dz;
      k1_antenna<T><<<1, 32, 0, s>>>(g, a, J + n);
      nl++;
    }
    // 5. current filter, Ampère + PML-E
    tbeg(1);
    const T* Ja = J;
    if (cfg.filter_J && P > 0) {
      FiltJob1<T> jb;
      for (int q = 0; q < 3; q++) { jb.src[q] = J + q * n; jb.dst[q] = Jf + q * n; jb.comp[q] = 6 + q; }
      k1_filter<T><<<dim3(nb1(n1, 256), 3), 256, 0, s>>>(g, jb, taps);
      nl++;
      Ja = Jf;
    }
    k1_ampere<T><<<nb1(n1, 256), 256, 0, s>>>(g, pm, E, B, Ja, T(g.dt), T(kC * kC * g.idz), T(1.0 / kEps0));
    nl++;
    tend(1);
    step++;
    // 6. ion rows that left, plasma rows entering through z_hi
    if (loaded) {
      while (mlo < row_next && (mlo + 0.5) * lat.h - beta * kC * tn1 < z_lo()) mlo++;
      const long long m_end = rows_inside(tn1);
      if (m_end > row_next) {
        if (inject(row_next, m_end, tn1) != PIC_OK) return st;
        row_next = m_end;
      }
      // the dead slots (left the domain, or rows without plasma) are squeezed out now and then
      if (count_ub > 65536 && (step & 63) == 0) {
        if (compact() != PIC_OK) return st;
      }
    }
    return PIC_OK;
  }

  int run(int nsteps) override {
    if (st != PIC_OK) return st;
    for (int q = 0; q < nsteps; q++)
      if (one_step() != PIC_OK) return st;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in 1D step");
  }

  int sync() override {
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PIC_ECUDA, "CUDA error");
    return st;
  }

  int btd_set(const pic_btd_req*) override { return fail(PIC_EINVAL, "1D: no boosted-to-lab samples"); }
  int btd_get(pic_btd_out*) override { return fail(PIC_EINVAL, "1D: no boosted-to-lab samples"); }

  T* comp_ptr(int comp) {
    const int n = g.n1p;
    if (comp < 3) return E + comp * n;
    if (comp < 6) return B + (comp - 3) * n;
    return J + (comp - 6) * n;
  }

  int get_field(int comp, double* dst, int on_device) override {
    if (comp < 0 || comp > PIC_RHO) return fail(PIC_EINVAL, "bad component");
    const int n1 = g.nz + 1;
    if (comp == PIC_RHO) {
      cudaMemsetAsync(rho, 0, sizeof(double) * g.n1p, s);
      if (loaded && count_ub > 0) {
        k1_rho_e<T><<<nb1(count_ub, 128), 128, 0, s>>>(g, P2[cur], ctrl, cfg.shape_order, rho);
        nl++;
      }
      if (loaded && ions && row_next > mlo) {
        k1_rho_i<<<nb1(n1, 128), 128, 0, s>>>(g, lat, cfg.shape_order, mlo, row_next, time_of(step), rho);
        nl++;
      }
      cudaMemcpyAsync(dst, rho, sizeof(double) * n1, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    } else {
      k1_out<T><<<nb1(n1, 256), 256, 0, s>>>(n1, comp_ptr(comp), outd);
      nl++;
      cudaMemcpyAsync(dst, outd, sizeof(double) * n1, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    }
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in get_field");
  }

  int set_field(int comp, const double* src) override {
    if (comp < 0 || comp > 8) return fail(PIC_EINVAL, "bad component");
    const int n1 = g.nz + 1;
    cudaMemcpyAsync(outd, src, sizeof(double) * n1, cudaMemcpyHostToDevice, s);
    k1_in<T><<<nb1(n1, 256), 256, 0, s>>>(n1, outd, comp_ptr(comp));
    nl++;
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in set_field");
  }

  int get_particles(int species, double* x, double* y, double* z, double* ux, double* uy, double* uz, double* w,
                    uint32_t* id, int32_t* flags, int64_t* count) override {
    if (species != 0) return fail(PIC_EINVAL, "1D: electrons only (the ions are a column current)");
    if (!loaded) { if (count) *count = 0; return PIC_OK; }
    // live electrons in slot order
    const int c = read_count();
    if (c < 0) return fail(PIC_ECUDA, "CUDA error");
    std::vector<double> hz(c);
    std::vector<T> hux(c), huy(c), huz(c), hw(c);
    std::vector<uint32_t> hid(c);
    const Parts1<T>& p = P2[cur];
    if (c > 0) {
      cudaMemcpyAsync(hz.data(), p.z, 8 * (size_t)c, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hux.data(), p.ux, sizeof(T) * c, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(huy.data(), p.uy, sizeof(T) * c, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(huz.data(), p.uz, sizeof(T) * c, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hw.data(), p.w, sizeof(T) * c, cudaMemcpyDeviceToHost, s);
      cudaMemcpyAsync(hid.data(), p.id, 4 * (size_t)c, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PIC_ECUDA, "CUDA error");
    }
    int64_t o = 0;
    const bool want = x || y || z || ux || uy || uz || w || id || flags;
    for (int j = 0; j < c; j++) {
      if (!(hw[j] > T(0))) continue;
      if (want) {
        if (x) x[o] = 0.0;
        if (y) y[o] = 0.0;
        if (z) z[o] = hz[j];
        if (ux) ux[o] = (double)hux[j];
        if (uy) uy[o] = (double)huy[j];
        if (uz) uz[o] = (double)huz[j];
        if (w) w[o] = (double)hw[j];
        if (id) id[o] = hid[j];
        if (flags) flags[o] = 1;
      }
      o++;
    }
    if (count) *count = o;
    return PIC_OK;
  }

  int stats(pic_stats* o) override {
    double trap = o->trap_gamma_lab > 0.0 ? o->trap_gamma_lab : 0.0;
    if (trap == 0.0 && has_laser && loaded && lat.n0 > 0.0) {
      const double wp = std::sqrt(lat.n0 * kQe * kQe / (kEps0 * kMe));
      trap = 2.0 * (2.0 * kPi * kC / las.lambda0) / wp;
    }
    cudaMemsetAsync(sred, 0, 4 * sizeof(double), s);
    Parts1<T> p = P2[cur];
    if (!loaded) cudaMemsetAsync(ctrl, 0, sizeof(Ctrl1), s);
    k1_stats<T><<<64, 256, 0, s>>>(g, E, B, p, ctrl, gamma, beta, trap, sred);
    nl++;
    double h[4];
    cudaMemcpyAsync(h, sred, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PIC_ECUDA, "CUDA error in stats");
    o->step = step; o->t = time_of(step);
    o->dt = g.dt; o->dx = 0.0; o->dz = g.dz; o->gamma = gamma; o->beta = beta;
    o->n_electrons = loaded ? (int64_t)h[0] : 0;
    o->n_beam_active = 0; o->beam_gamma_lab = 0.0; o->beam_spread = 0.0;
    o->field_energy = h[1];
    o->gx_lo = 0; o->gx_hi = 0; o->gz_lo = g.lo; o->gz_hi = g.hi;
    o->sorts = compactions; o->overflow_chunks = 0;
    o->z0 = g.z0;
    o->trap_gamma_lab = trap;
    o->trapped_charge = kQe * h[2];
    return PIC_OK;
  }

  int64_t launches() const override { return nl; }

  int kernel_timing(int enable, int which, double* ms_total, int64_t* n) override {
    if (which != 0 && which != 1) return PIC_EINVAL;
    if (!ev0) { cudaEventCreate(&ev0); cudaEventCreate(&ev1); }
    tcollect();
    if (enable >= 0) {
      timing_on = enable != 0;
      timing_which = which;
      if (enable) { t_ms = 0; t_n = 0; }
    }
    if (ms_total) *ms_total = t_ms;
    if (n) *n = t_n;
    return PIC_OK;
  }

  int status() const override { return st; }
  const std::string& error() const override { return err; }

 private:
  pic_config cfg;
  pic_alloc_fn alloc;
  pic_free_fn freef;
  void* user;
  cudaStream_t s;
  std::vector<std::pair<void*, size_t>> allocs;
  int st = PIC_OK;
  std::string err;
  G1 g{};
  double gamma = 1.0, beta = 0.0;
  int P = 0;
  bool nodal = false;
  Taps1<T> taps{};
  Pml1<T> pm{};
  T *E = nullptr, *B = nullptr, *J = nullptr, *Jf = nullptr, *Ep = nullptr, *Eb = nullptr, *Bavg = nullptr;
  T *fE = nullptr, *fB = nullptr, *nF = nullptr;
  double *rho = nullptr, *outd = nullptr, *sred = nullptr;
  Ctrl1* ctrl = nullptr;
  T** shift_arr = nullptr;
  int* shift_comp = nullptr;
  Parts1<T> P2[2]{};
  int cur = 0;
  int* blk = nullptr;
  long cap = 0;
  long count_ub = 0, live_est = 0;
  bool loaded = false, ions = false, has_laser = false;
  Lat1 lat{};
  pic_laser las{};
  long long row_next = 0, mlo = 0, shifts = 0, step = 0;
  int64_t nl = 0, compactions = 0;
  bool timing_on = false;
  int timing_which = 0;
  double t_ms = 0;
  std::vector<cudaEvent_t> tev;
  int64_t t_n = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

}  // namespace

Sim3Api* make_sim1(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* user, cudaStream_t s,
                   int* status, std::string* err) {
  Sim3Api* r = nullptr;
  int st = PIC_OK;
  if (cfg->precision == PIC_FP64) {
    auto* p = new Sim1<double>(*cfg, alloc, free_fn, user, s);
    st = p->init();
    if (st != PIC_OK) { if (err) *err = p->error(); delete p; } else r = p;
  } else {
    auto* p = new Sim1<float>(*cfg, alloc, free_fn, user, s);
    st = p->init();
    if (st != PIC_OK) { if (err) *err = p->error(); delete p; } else r = p;
  }
  if (status) *status = st;
  return r;
}

}  // namespace picgb
