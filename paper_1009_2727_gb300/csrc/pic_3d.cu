// 3D (x, y, z) boosted-frame PIC step on the GPU: the same method as the
// 2-1/2D path, written for three dimensions (Vay et al., arXiv:1009.2727).
//  - Faraday with the enlarged operator of Sec. 4.2, Delta*_a = (alpha +
//    beta S1 + gamma S2) Delta_a, S1/S2 the transverse neighbours one full
//    cell away (PR-2), Friedman E_eff (Eq. Faraday_Friedman), split-field PML
//    on all six faces (App. II): each component is the sum of two parts, one
//    per derivative direction, each damped by its own axis' sigma.
//  - Ampere with the Yee operator and the same split PML.
//  - Composed multi-pass bilinear filter per axis (Sec. 4.1) on the current
//    and on the gathered fields.
//  - Energy-conserving gather from the Yee positions with linear or cubic
//    B-splines, Boris push, 3D Esirkepov deposition (Esirkepov 2001).
//  - Cold plasma through the +z plane on a ppc_x x ppc_y x ppc_z lattice,
//    rigid ions fixed in the lab as a separable column current; the laser
//    from dual particle arrays (Sec. 3.1.2), one pair per transverse node
//    whose moving partner is displaced along y and deposits with Esirkepov.
//  - Test beam through a plane, lab-frame samples (Sec. 3.2), diagnostics.
// Layout: node (i,j,k) of every component at (i*(ny+1)+j)*ldz + k, ldz the
// padded z extent; Ex (i+1/2,j,k), Ey (i,j+1/2,k), Ez (i,j,k+1/2),
// Bx (i,j+1/2,k+1/2), By (i+1/2,j,k+1/2), Bz (i+1/2,j+1/2,k); J like E.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pic_3d.h"
#include "pic_common.cuh"

namespace picgb {
namespace {

struct G3 {
  int n[3];        // cells along x, y, z
  int ldz;         // padded z extent of every array
  long cs;         // elements per component array
  double d[3];     // cell sizes
  double id[3];    // their inverses (host division, so the sweeps run no FP64 divide)
  double dt;
  int lo[3], hi[3];  // particle domain [cells]
};

__host__ __device__ inline long nid(const G3& g, int i, int j, int k) {
  return ((long)i * (g.n[1] + 1) + j) * g.ldz + k;
}

inline unsigned nblk(long n, int b) { return (unsigned)((n + b - 1) / b); }

// valid index range of component c (0..5: E then B; J uses E) along an axis: half-staggered 0..n-1,
// integer 1..n-1 for E (tangential E vanishes on the PEC walls) and 0..n for B
__host__ __device__ inline void vr(int c, int axis, const G3& g, int& lo, int& hi) {
  const int n = g.n[axis];
  const bool half = c < 3 ? (c == axis) : (c - 3 != axis);
  if (half) { lo = 0; hi = n - 1; }
  else if (c < 3) { lo = 1; hi = n - 1; }
  else { lo = 0; hi = n; }
}

__host__ __device__ inline bool in_valid(int c, const G3& g, int i, int j, int k) {
  int lo, hi;
  vr(c, 0, g, lo, hi); if (i < lo || i > hi) return false;
  vr(c, 1, g, lo, hi); if (j < lo || j > hi) return false;
  vr(c, 2, g, lo, hi); if (k < lo || k > hi) return false;
  return true;
}

template <class T>
__device__ __forceinline__ T rd3(const G3& g, const T* F, int i, int j, int k) {
  if (i < 0 || i > g.n[0] || j < 0 || j > g.n[1] || k < 0 || k > g.n[2]) return T(0);
  return F[nid(g, i, j, k)];
}

__device__ __forceinline__ bool node_of(const G3& g, long p, int& i, int& j, int& k) {
  const long nz1 = g.n[2] + 1, ny1 = g.n[1] + 1;
  if (p >= (long)(g.n[0] + 1) * ny1 * nz1) return false;
  k = (int)(p % nz1);
  const long r = p / nz1;
  j = (int)(r % ny1);
  i = (int)(r / ny1);
  return true;
}

// PML tables per axis at integer and half positions, in the path's own real type: the FP64 path keeps them
// in FP64; the mixed path rounds them to FP32 once (on this GPU an FP64 operation per PML node and
// component would make the field sweeps FP64-pipe bound)
template <class T>
struct Pml3 {
  const T* sg[3][2];   // sigma [axis][half]
  const T* xi[3][2];
  const T* cf[3][2];   // (1 - xi)/sigma, dt where sigma = 0
  T id[3];             // inverse cell sizes in the path's type (no FP64 conversion in the sweeps)
};

// current per unit weight of the push, -q d_a/(d_x d_y d_z dt) per axis, computed on the host
template <class T>
struct Cq3 {
  T v[3];
};

struct Ctrl3 {
  int count;
  int status;
  int pad[2];
  double red[8];
};

template <class T>
struct Taps3 {
  T c[2 * FILTER_HMAX + 1];
  int P, s;
};

// ---------------------------------------------------------------------------
// fields
// Faraday with the enlarged operator, Friedman's E_eff and the split PML for B (PR-1, PR-2), over a tile
// of FX x FY x FZ nodes. E_eff = c1 E^n - c2 E^{n-1} + c3 E-bar^{n-2} is formed while the tile and a
// one-node halo are staged in shared memory (zero off the grid); each thread then updates the three B
// components of FX nodes along x.
//   Delta*_a F at a node (result half a cell above along a) = (alpha D(0,0) + beta (four axial neighbours)
//   + gamma (four diagonal neighbours)) / d_a, D the difference along a on the transverse offsets.
constexpr int FX = 4, FY = 8, FZ = 32;
// z nodes per thread of the other grid sweeps (a block width apart)
constexpr int KPT = 4;

template <class T>
__device__ __forceinline__ T dstar_s(const T* S, int a, int c0, T ca, T cb, T cg, T inv_d) {
  constexpr int SY = FY + 2, SZ = FZ + 2;
  constexpr int st[3] = {SY * SZ, SZ, 1};
  const int b = a == 0 ? 1 : 0, c = a == 2 ? 1 : 2;
  T D[3][3];
#pragma unroll
  for (int o1 = -1; o1 <= 1; o1++)
#pragma unroll
    for (int o2 = -1; o2 <= 1; o2++) {
      const int q = c0 + o1 * st[b] + o2 * st[c];
      D[o1 + 1][o2 + 1] = S[q + st[a]] - S[q];
    }
  const T s1 = D[0][1] + D[2][1] + D[1][0] + D[1][2];
  const T s2 = D[0][0] + D[0][2] + D[2][0] + D[2][2];
  return (ca * D[1][1] + cb * s1 + cg * s2) * inv_d;
}

template <class T>
__global__ void __launch_bounds__(256) k3_faraday_tile(G3 g, Pml3<T> pm, const T* __restrict__ E,
                                                       const T* __restrict__ Ep, const T* __restrict__ Eb,
                                                       T* __restrict__ B, T* __restrict__ Bs, T* __restrict__ fB, T c1,
                                                       T c2, T c3, T ca, T cb, T cg, T dtT) {
  constexpr int SX = FX + 2, SY = FY + 2, SZ = FZ + 2, SN = SX * SY * SZ;
  __shared__ T se[3][SN];   // index (x * SY + y) * SZ + z, tile origin at (1, 1, 1)
  const int i0 = blockIdx.z * FX, j0 = blockIdx.y * FY, k0 = blockIdx.x * FZ;
  const int tid = threadIdx.y * FZ + threadIdx.x;
  for (int e = tid; e < SN; e += FZ * FY) {
    const int lz = e % SZ, r = e / SZ, ly = r % SY, lx = r / SY;
    const int i = i0 - 1 + lx, j = j0 - 1 + ly, k = k0 - 1 + lz;
    if (i >= 0 && i <= g.n[0] && j >= 0 && j <= g.n[1] && k >= 0 && k <= g.n[2]) {
      const long p = nid(g, i, j, k);
#pragma unroll
      for (int q = 0; q < 3; q++) se[q][e] = c1 * E[q * g.cs + p] - c2 * Ep[q * g.cs + p] + c3 * Eb[q * g.cs + p];
    } else {
#pragma unroll
      for (int q = 0; q < 3; q++) se[q][e] = T(0);
    }
  }
  __syncthreads();
  const int j = j0 + threadIdx.y, k = k0 + threadIdx.x;
  if (j > g.n[1] || k > g.n[2]) return;
#pragma unroll
  for (int lx = 0; lx < FX; lx++) {
    const int i = i0 + lx;
    if (i > g.n[0]) break;
    const long p = nid(g, i, j, k);
    const int c0 = ((lx + 1) * SY + threadIdx.y + 1) * SZ + threadIdx.x + 1;
    const int idx[3] = {i, j, k};
    const bool in = i >= 1 && i < g.n[0] && j >= 1 && j < g.n[1] && k >= 1 && k < g.n[2];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const T old = B[q * g.cs + p];
      T nw = old;
      // every B component is valid on the interior nodes
      if (in || in_valid(3 + q, g, i, j, k)) {
        const int u = (q + 1) % 3, v = (q + 2) % 3;
        const T du = dstar_s<T>(se[v], u, c0, ca, cb, cg, pm.id[u]);
        const T dv = dstar_s<T>(se[u], v, c0, ca, cb, cg, pm.id[v]);
        const T su = pm.sg[u][1][idx[u]], sv = pm.sg[v][1][idx[v]];
        if (su > T(0) || sv > T(0)) {
          T* Pu = Bs + (2 * q) * g.cs;
          T* Pv = Bs + (2 * q + 1) * g.cs;
          const T a = pm.xi[u][1][idx[u]] * Pu[p] - pm.cf[u][1][idx[u]] * du;
          const T b = pm.xi[v][1][idx[v]] * Pv[p] + pm.cf[v][1][idx[v]] * dv;
          Pu[p] = a;
          Pv[p] = b;
          nw = a + b;
        } else {
          nw = old - dtT * (du - dv);
        }
        B[q * g.cs + p] = nw;
      }
      fB[q * g.cs + p] = T(0.5) * (old + nw);
    }
  }
}

// Friedman history (PR-1): E-bar <- (1 - theta/2) E + (theta/2) E-bar, E^{n-1} <- E, gather copy <- E
template <class T>
__global__ void k3_friedman(long n, const T* E, T* Ep, T* Eb, T* fE, T a, T b) {
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const T e = E[p];
  Eb[p] = a * e + b * Eb[p];
  Ep[p] = e;
  fE[p] = e;
}

template <class T>
__device__ __forceinline__ void ampere_node(const G3& g, const Pml3<T>& pm, T* __restrict__ E, T* __restrict__ Es,
                                            const T* __restrict__ B, const T* __restrict__ J, T dtc2, T dte, int i,
                                            int j, int k) {
  const long p = nid(g, i, j, k);
  const int idx[3] = {i, j, k};
  const T c2 = T(kC * kC);
  const bool in = i >= 1 && j >= 1 && k >= 1;
  // E is valid off the PEC walls: 1..n-1 on integer axes, 0..n-1 on its own half axis
  const bool allv = in && i < g.n[0] && j < g.n[1] && k < g.n[2];
  const long st[3] = {(long)(g.n[1] + 1) * g.ldz, g.ldz, 1};
#pragma unroll
  for (int q = 0; q < 3; q++) {
    if (!allv && !in_valid(q, g, i, j, k)) continue;
    const int u = (q + 1) % 3, v = (q + 2) % 3;
    // dE_q/dt = c^2 (Delta_u B_v - Delta_v B_u) - J_q/eps0, backward differences
    const T* Bv = B + v * g.cs;
    const T* Bu = B + u * g.cs;
    T du, dv;
    if (in) {
      du = (Bv[p] - Bv[p - st[u]]) * pm.id[u];
      dv = (Bu[p] - Bu[p - st[v]]) * pm.id[v];
    } else {
      du = (rd3(g, Bv, i, j, k) - rd3(g, Bv, i - (u == 0), j - (u == 1), k - (u == 2))) * pm.id[u];
      dv = (rd3(g, Bu, i, j, k) - rd3(g, Bu, i - (v == 0), j - (v == 1), k - (v == 2))) * pm.id[v];
    }
    const T su = pm.sg[u][0][idx[u]], sv = pm.sg[v][0][idx[v]];
    if (su > T(0) || sv > T(0)) {
      T* Pu = Es + (2 * q) * g.cs;
      T* Pv = Es + (2 * q + 1) * g.cs;
      const T a = pm.xi[u][0][idx[u]] * Pu[p] + c2 * pm.cf[u][0][idx[u]] * du;
      const T b = pm.xi[v][0][idx[v]] * Pv[p] - c2 * pm.cf[v][0][idx[v]] * dv;
      Pu[p] = a;
      Pv[p] = b;
      E[q * g.cs + p] = a + b;
    } else {
      E[q * g.cs + p] = E[q * g.cs + p] + (dtc2 * (du - dv) - dte * J[q * g.cs + p]);
    }
  }
}

template <class T>
__global__ void __launch_bounds__(128) k3_ampere(G3 g, Pml3<T> pm, T* __restrict__ E, T* __restrict__ Es,
                                                 const T* __restrict__ B, const T* __restrict__ J, T dtc2, T dte) {
  const int k0 = blockIdx.x * blockDim.x * KPT + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
#pragma unroll
  for (int kk = 0; kk < KPT; kk++) {
    const int k = k0 + kk * blockDim.x;
    if (k > g.n[2]) break;
    ampere_node<T>(g, pm, E, Es, B, J, dtc2, dte, i, j, k);
  }
}

// one axis of the composed filter: out = sum_m c_m F(node + (m - P) s e_axis), zero off the valid range.
// PT > 0: the pass count P is the template constant (taps unrolled); PT = 0: any P. Each thread filters
// KPT z nodes a block width apart (coalesced).
template <class T, int PT>
__global__ void __launch_bounds__(128) k3_filter_axis(G3 g, const T* __restrict__ src, T* __restrict__ dst, int comp,
                                                      int axis, Taps3<T> t) {
  const int k0 = blockIdx.x * blockDim.x * KPT + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  if (k0 > g.n[2]) return;
  const int P = PT > 0 ? PT : t.P;
  const long st = axis == 0 ? (long)(g.n[1] + 1) * g.ldz : axis == 1 ? (long)g.ldz : 1L;
  const int R = P * t.s;
  const long ss = st * t.s;
  const int n = g.n[axis];
#pragma unroll
  for (int kk = 0; kk < KPT; kk++) {
    const int k = k0 + kk * blockDim.x;
    if (k > g.n[2]) break;
    const long p = nid(g, i, j, k);
    if (!in_valid(comp, g, i, j, k)) {
      dst[p] = T(0);
      continue;
    }
    const int id = axis == 0 ? i : axis == 1 ? j : k;
    const T* q0 = src + p - R * st;
    T acc = T(0);
    if (id - R >= 0 && id + R <= n) {
      if (PT > 0) {
#pragma unroll
        for (int m = 0; m <= 2 * PT; m++) acc += t.c[m] * q0[m * ss];
      } else {
        for (int m = 0; m <= 2 * P; m++) acc += t.c[m] * q0[m * ss];
      }
    } else {
      for (int m = 0; m <= 2 * P; m++) {
        const int o = id + (m - P) * t.s;
        if (o >= 0 && o <= n) acc += t.c[m] * q0[m * ss];
      }
    }
    dst[p] = acc;
  }
}

// x or y axis of the composed filter (stride 1, PT taps each side): a register window slides along the
// axis; each thread owns one segment of one line (one z node, one index of the other transverse axis,
// nodes [a, b) along the axis), reads each node of the segment and its 2 PT neighbours once, and sums the
// taps in the same order as k3_filter_axis. Nodes off the grid read as zero.
template <class T, int PT>
__global__ void __launch_bounds__(128) k3_filter_slide(G3 g, const T* __restrict__ src, T* __restrict__ dst, int comp,
                                                       int axis, int seg, Taps3<T> t) {
  constexpr int W = 2 * PT + 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x, o = blockIdx.y;
  if (k > g.n[2]) return;
  const int n = axis == 0 ? g.n[0] : g.n[1];
  const int a = blockIdx.z * seg, b = min(a + seg, n + 1);
  int lo0, hi0, lo1, hi1, lo2, hi2;
  vr(comp, 0, g, lo0, hi0);
  vr(comp, 1, g, lo1, hi1);
  vr(comp, 2, g, lo2, hi2);
  const int loa = axis == 0 ? lo0 : lo1, hia = axis == 0 ? hi0 : hi1;
  const bool other = (axis == 0 ? (o >= lo1 && o <= hi1) : (o >= lo0 && o <= hi0)) && k >= lo2 && k <= hi2;
  const long st = axis == 0 ? (long)(g.n[1] + 1) * g.ldz : (long)g.ldz;
  const long base = axis == 0 ? nid(g, 0, o, k) : nid(g, o, 0, k);
  T c[W];
#pragma unroll
  for (int m = 0; m < W; m++) c[m] = t.c[m];
  // w[m] = src at index i - PT + m
  T w[W];
#pragma unroll
  for (int m = 0; m < W; m++) {
    const int q = a + m - PT;
    w[m] = (q >= 0 && q <= n) ? src[base + q * st] : T(0);
  }
  for (int i0 = a; i0 < b; i0 += W) {
#pragma unroll
    for (int r = 0; r < W; r++) {
      const int i = i0 + r;
      if (i < b) {
        T acc = T(0);
#pragma unroll
        for (int m = 0; m < W; m++) acc += c[m] * w[m];
        dst[base + i * st] = (other && i >= loa && i <= hia) ? acc : T(0);
      }
#pragma unroll
      for (int m = 0; m < W - 1; m++) w[m] = w[m + 1];
      const int q = i + PT + 1;
      w[W - 1] = (i + 1 < b && q <= n) ? src[base + q * st] : T(0);
    }
  }
}

// 16-byte shared-memory load of 16 / sizeof(T) consecutive values
__device__ __forceinline__ void ld16(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
}
__device__ __forceinline__ void ld16(const double* p, double* v) {
  const double2 q = *reinterpret_cast<const double2*>(p);
  v[0] = q.x; v[1] = q.y;
}

// z axis of the composed filter (stride 1): each block stages a row segment of 128 * ZR nodes and an
// 8-node halo in shared memory; each thread reads its ZR + 16 staged values with 16-byte loads and sums
// the taps of ZR consecutive outputs in the same order as k3_filter_axis.
// A row's last block also takes a remainder of up to ZTAIL nodes past its segment (a row of 2^m + 1 nodes
// would otherwise need a block for its last node); longer remainders get a block of their own.
constexpr int ZR = 8, ZHA = 8, ZTAIL = 32;
template <class T, int PT>
__global__ void __launch_bounds__(128) k3_filter_zs(G3 g, const T* __restrict__ src, T* __restrict__ dst, int comp,
                                                    Taps3<T> t) {
  static_assert(PT <= ZHA, "filter halo above the staged halo");
  constexpr int SEG = 128 * ZR, NV = ZR + 2 * ZHA, VL = 16 / (int)sizeof(T);
  constexpr int ROW = SEG + 2 * ZHA + ZTAIL, NVEC = ROW / VL, UV = (NVEC + 127) / 128;
  static_assert(ROW % VL == 0 && ZHA % VL == 0, "16-byte vectors tile the staged row");
  typedef typename std::conditional<sizeof(T) == 4, float4, double2>::type V;
  __shared__ __align__(16) T row[ROW];
  const int kb = blockIdx.x * SEG, j = blockIdx.y, i = blockIdx.z;
  const int n = g.n[2];
  // nodes past this segment that this block also filters (the row's last block only)
  const int tail = blockIdx.x + 1 == gridDim.x ? min(max(n + 1 - (kb + SEG), 0), ZTAIL) : 0;
  const long base = nid(g, i, j, 0);   // 16-byte aligned: ldz is padded to 128 bytes
  // the staged row in 16-byte vectors, every thread's loads issued before any is stored (an element
  // q of the row is node kb - ZHA + q; off the row: zero)
  V vv[UV];
#pragma unroll
  for (int u = 0; u < UV; u++) {
    const int e = (threadIdx.x + u * 128) * VL, q0 = kb - ZHA + e;
    T x[VL];
#pragma unroll
    for (int l = 0; l < VL; l++) x[l] = T(0);
    if (e < SEG + 2 * ZHA + tail) {
      if (q0 >= 0 && q0 + VL - 1 <= n) {
        const V w = *reinterpret_cast<const V*>(src + base + q0);
        if constexpr (VL == 4) { x[0] = w.x; x[1] = w.y; x[2] = w.z; x[3] = w.w; }
        else { x[0] = w.x; x[1] = w.y; }
      } else {
#pragma unroll
        for (int l = 0; l < VL; l++)
          if (q0 + l >= 0 && q0 + l <= n) x[l] = src[base + q0 + l];
      }
    }
    if constexpr (VL == 4) vv[u] = make_float4(x[0], x[1], x[2], x[3]);
    else vv[u] = make_double2(x[0], x[1]);
  }
#pragma unroll
  for (int u = 0; u < UV; u++) {
    const int vi = threadIdx.x + u * 128;
    if (vi < NVEC) reinterpret_cast<V*>(row)[vi] = vv[u];
  }
  __syncthreads();
  int lo0, hi0, lo1, hi1, lo2, hi2;
  vr(comp, 0, g, lo0, hi0);
  vr(comp, 1, g, lo1, hi1);
  vr(comp, 2, g, lo2, hi2);
  const bool other = i >= lo0 && i <= hi0 && j >= lo1 && j <= hi1;
  const int l0 = ZR * threadIdx.x;
  T v[NV];
#pragma unroll
  for (int q = 0; q < NV / VL; q++) ld16(row + l0 + q * VL, v + q * VL);
  T o[ZR];
#pragma unroll
  for (int r = 0; r < ZR; r++) {
    const int k = kb + l0 + r;
    T acc = T(0);
#pragma unroll
    for (int m = 0; m <= 2 * PT; m++) acc += t.c[m] * v[r + ZHA - PT + m];
    o[r] = (other && k >= lo2 && k <= hi2) ? acc : T(0);
  }
  if (kb + l0 + ZR - 1 <= n) {
#pragma unroll
    for (int r = 0; r < ZR; r += VL) {
      V w;
      if constexpr (VL == 4) w = make_float4(o[r], o[r + 1], o[r + 2], o[r + 3]);
      else w = make_double2(o[r], o[r + 1]);
      *reinterpret_cast<V*>(dst + base + kb + l0 + r) = w;
    }
  } else {
#pragma unroll
    for (int r = 0; r < ZR; r++)
      if (kb + l0 + r <= n) dst[base + kb + l0 + r] = o[r];
  }
  if ((int)threadIdx.x < tail) {
    const int e = SEG + threadIdx.x, k = kb + e;   // k <= n by the choice of tail
    T acc = T(0);
#pragma unroll
    for (int m = 0; m <= 2 * PT; m++) acc += t.c[m] * row[e + ZHA - PT + m];
    dst[base + k] = (other && k >= lo2 && k <= hi2) ? acc : T(0);
  }
}

// blocks along a row of n + 1 nodes for k3_filter_zs: a remainder of up to ZTAIL nodes rides with the last
// segment
inline unsigned zs_blocks(int n) {
  constexpr int SEG = 128 * ZR;
  const int full = (n + 1) / SEG, rem = n + 1 - full * SEG;
  return (unsigned)(full == 0 ? 1 : full + (rem > ZTAIL ? 1 : 0));
}

// x and y axes of the composed filter (stride 1, PT taps each side) in one pass. A CTA stages, by one bulk
// tensor copy, a box of the source (XYT + 2 PT nodes along x and along y, ZB along z; off-grid nodes arrive
// as zero), filters it along x into a scratch box that keeps the y halo, then along y, and writes the
// XYT x XYT x ZB outputs: one read and one write of the component instead of two of each. Each thread
// slides a register window along its line, summing the taps in the same order as k3_filter_axis, and the
// outputs of either pass at invalid nodes of the component are zero, as in the separate sweeps.
constexpr int XYT = 16, ZB = 16;
constexpr long kWait3 = 1L << 24;

template <class T, int PT>
__global__ void __launch_bounds__(256) k3_filter_xy(G3 g, const __grid_constant__ CUtensorMap map, int slot,
                                                    T* __restrict__ dst, int comp, Taps3<T> t, Ctrl3* ctrl) {
  constexpr int W = 2 * PT + 1, XW = XYT + 2 * PT;
  extern __shared__ __align__(128) unsigned char raw3[];
  T* S = reinterpret_cast<T*>(raw3 + ((128u - ((uint32_t)__cvta_generic_to_shared(raw3) & 127u)) & 127u));
  // after the x pass: [x 0..XYT) [y 0..XW) [z 0..ZB), x planes XP apart (padded by 16 elements, so that the
  // two x planes a warp of the y pass reads fall in different banks)
  constexpr int XP = XW * ZB + 16;
  T* X1 = S + XW * XW * ZB;
  __shared__ __align__(8) uint64_t bar;
  const int k0 = blockIdx.x * ZB, j0 = blockIdx.y * XYT, i0 = blockIdx.z * XYT;
  const int tid = threadIdx.x;
  const uint32_t sbar = (uint32_t)__cvta_generic_to_shared(&bar);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar),
                 "r"((uint32_t)(XW * XW * ZB * sizeof(T)))
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"((uint32_t)__cvta_generic_to_shared(S)),
        "l"((unsigned long long)&map), "r"(k0), "r"(j0 - PT), "r"(i0 - PT), "r"(slot), "r"(sbar)
        : "memory");
  }
  // one warp polls the mbarrier; the others wait at the barrier below, taking no issue slots
  bool done = tid >= 32;
  for (long it = 0; it < kWait3 && !done; it++) {
    uint32_t d;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(d)
        : "r"(sbar)
        : "memory");
    done = d != 0;
  }
  // the outcome is made block-uniform; a timed-out block records it and leaves once its copy has landed
  if (__syncthreads_or(!done)) {
    if (tid == 0) {
      atomicOr(&ctrl->status, (int)ST_TIMEOUT);
      for (long it = 0; it < kWait3; it++) {
        uint32_t d;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(d)
            : "r"(sbar)
            : "memory");
        if (d) break;
      }
    }
    return;
  }
  int lo0, hi0, lo1, hi1, lo2, hi2;
  vr(comp, 0, g, lo0, hi0);
  vr(comp, 1, g, lo1, hi1);
  vr(comp, 2, g, lo2, hi2);
  T c[W];
#pragma unroll
  for (int m = 0; m < W; m++) c[m] = t.c[m];
  // x pass: one (y, z) line of the box per task, XYT outputs
  for (int task = tid; task < XW * ZB; task += 256) {
    const int yi = task / ZB, zi = task - yi * ZB;
    const int gj = j0 - PT + yi, gk = k0 + zi;
    const bool other = gj >= lo1 && gj <= hi1 && gk >= lo2 && gk <= hi2;
    const T* col = S + yi * ZB + zi;
    T w[W];
#pragma unroll
    for (int m = 0; m < W; m++) w[m] = col[m * XW * ZB];
#pragma unroll
    for (int xo = 0; xo < XYT; xo++) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < W; m++) acc += c[m] * w[m];
      const int gi = i0 + xo;
      X1[xo * XP + yi * ZB + zi] = (other && gi >= lo0 && gi <= hi0) ? acc : T(0);
      if (xo + 1 < XYT) {
#pragma unroll
        for (int m = 0; m < W - 1; m++) w[m] = w[m + 1];
        w[W - 1] = col[(xo + W) * XW * ZB];
      }
    }
  }
  __syncthreads();
  // y pass: one (x, z) line per thread, XYT outputs written to dst
  {
    const int xo = tid / ZB, zi = tid - xo * ZB;
    const int gi = i0 + xo, gk = k0 + zi;
    const bool other = gi >= lo0 && gi <= hi0 && gk >= lo2 && gk <= hi2;
    const bool in = gi <= g.n[0] && gk <= g.n[2];
    const T* row = X1 + xo * XP + zi;
    T w[W];
#pragma unroll
    for (int m = 0; m < W; m++) w[m] = row[m * ZB];
#pragma unroll
    for (int yo = 0; yo < XYT; yo++) {
      T acc = T(0);
#pragma unroll
      for (int m = 0; m < W; m++) acc += c[m] * w[m];
      const int gj = j0 + yo;
      if (in && gj <= g.n[1]) dst[nid(g, gi, gj, gk)] = (other && gj >= lo1 && gj <= hi1) ? acc : T(0);
      if (yo + 1 < XYT) {
#pragma unroll
        for (int m = 0; m < W - 1; m++) w[m] = w[m + 1];
        w[W - 1] = row[(yo + W) * ZB];
      }
    }
  }
}
static_assert(XYT * ZB == 256, "one y-pass line per thread");

template <class T, int PT>
constexpr size_t filter_xy_smem() {
  return (size_t)((XYT + 2 * PT) * (XYT + 2 * PT) * ZB + XYT * ((XYT + 2 * PT) * ZB + 16)) * sizeof(T) + 128;
}

typedef CUresult (*Encode3Fn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// 4D tensor over a 3-component block (z, y, x, component), boxes of ZB x (XYT + 2 halo)^2 x 1 nodes, zero
// fill off the grid; false when the driver entry point is missing or the encoding is refused
template <class T>
bool encode_xy_map(CUtensorMap* m, const T* base, const G3& g, int halo) {
  static Encode3Fn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (Encode3Fn)p;
  }
  if (!fn || !base) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)(g.n[2] + 1), (cuuint64_t)(g.n[1] + 1), (cuuint64_t)(g.n[0] + 1), 3};
  const cuuint64_t strides[3] = {(cuuint64_t)g.ldz * sizeof(T), (cuuint64_t)(g.n[1] + 1) * g.ldz * sizeof(T),
                                 (cuuint64_t)g.cs * sizeof(T)};
  const cuuint32_t box[4] = {(cuuint32_t)ZB, (cuuint32_t)(XYT + 2 * halo), (cuuint32_t)(XYT + 2 * halo), 1};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, dt, 4, const_cast<T*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <class T, int PT>
void launch_filter_xy(const G3& g, const CUtensorMap& map, int slot, T* dst, int comp, const Taps3<T>& t,
                      Ctrl3* ctrl, cudaStream_t s) {
  const dim3 grid(nblk(g.n[2] + 1, ZB), nblk(g.n[1] + 1, XYT), nblk(g.n[0] + 1, XYT));
  k3_filter_xy<T, PT><<<grid, 256, filter_xy_smem<T, PT>(), s>>>(g, map, slot, dst, comp, t, ctrl);
}

template <class T>
void set_filter_xy_smem() {
  cudaFuncSetAttribute(k3_filter_xy<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_xy_smem<T, 1>());
  cudaFuncSetAttribute(k3_filter_xy<T, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_xy_smem<T, 2>());
  cudaFuncSetAttribute(k3_filter_xy<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_xy_smem<T, 3>());
  cudaFuncSetAttribute(k3_filter_xy<T, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_xy_smem<T, 4>());
  cudaFuncSetAttribute(k3_filter_xy<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filter_xy_smem<T, 5>());
}

template <class T, int PT>
void launch_filter_fast(const G3& g, const T* src, T* dst, int comp, int axis, const Taps3<T>& t, cudaStream_t s) {
  if (axis == 2) {
    k3_filter_zs<T, PT><<<dim3(zs_blocks(g.n[2]), g.n[1] + 1, g.n[0] + 1), 128, 0, s>>>(g, src, dst, comp, t);
  } else {
    // segments of about 32 nodes along the axis: enough lines in flight to cover the load latency
    const int n1 = (axis == 0 ? g.n[0] : g.n[1]) + 1;
    const int nseg = std::max(1, n1 / 32), seg = (n1 + nseg - 1) / nseg;
    k3_filter_slide<T, PT><<<dim3(nblk(g.n[2] + 1, 128), axis == 0 ? g.n[1] + 1 : g.n[0] + 1, nblk(n1, seg)), 128, 0,
                             s>>>(g, src, dst, comp, axis, seg, t);
  }
}

template <class T>
void launch_filter_axis(const G3& g, dim3 grid, const T* src, T* dst, int comp, int axis, const Taps3<T>& t,
                        cudaStream_t s) {
  if (t.s == 1) {
    switch (t.P) {
      case 1: launch_filter_fast<T, 1>(g, src, dst, comp, axis, t, s); return;
      case 2: launch_filter_fast<T, 2>(g, src, dst, comp, axis, t, s); return;
      case 3: launch_filter_fast<T, 3>(g, src, dst, comp, axis, t, s); return;
      case 4: launch_filter_fast<T, 4>(g, src, dst, comp, axis, t, s); return;
      case 5: launch_filter_fast<T, 5>(g, src, dst, comp, axis, t, s); return;
      default: break;
    }
  }
  switch (t.P) {
    case 1: k3_filter_axis<T, 1><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
    case 2: k3_filter_axis<T, 2><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
    case 3: k3_filter_axis<T, 3><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
    case 4: k3_filter_axis<T, 4><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
    case 5: k3_filter_axis<T, 5><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
    default: k3_filter_axis<T, 0><<<grid, 128, 0, s>>>(g, src, dst, comp, axis, t); break;
  }
}

// 'momentum conserving' gather (Sec. 5): node values of the six gather copies, the mean of the nearest
// staggered values along each half-integer axis of the component (two along one axis, four along two);
// values off the grid count as zero. dst holds Ex, Ey, Ez, Bx, By, Bz, cs elements each.
template <class T>
__global__ void __launch_bounds__(128) k3_nodal(G3 g, const T* __restrict__ fE, const T* __restrict__ fB,
                                                T* __restrict__ dst) {
  const int k0 = blockIdx.x * blockDim.x * KPT + threadIdx.x, j = blockIdx.y, i = blockIdx.z;
  const long sx = (long)(g.n[1] + 1) * g.ldz, sy = g.ldz;
#pragma unroll
  for (int kk = 0; kk < KPT; kk++) {
    const int k = k0 + kk * blockDim.x;
    if (k > g.n[2]) break;
    const long p = nid(g, i, j, k);
    const bool ok[3] = {i >= 1, j >= 1, k >= 1};
    const long st[3] = {sx, sy, 1};
#pragma unroll
    for (int c = 0; c < 6; c++) {
      // half-integer axes: E_q along q; B_q along the other two
      const int h0 = c < 3 ? (c == 0) : (c != 3), h1 = c < 3 ? (c == 1) : (c != 4), h2 = c < 3 ? (c == 2) : (c != 5);
      const T* F = (c < 3 ? fE + c * g.cs : fB + (c - 3) * g.cs) + p;
      const int h[3] = {h0, h1, h2};
      T acc = T(0);
      int cnt = 0;
#pragma unroll
      for (int a = 0; a <= 1; a++)
#pragma unroll
        for (int b = 0; b <= 1; b++)
#pragma unroll
          for (int e = 0; e <= 1; e++) {
            if ((a && !h[0]) || (b && !h[1]) || (e && !h[2])) continue;
            // neighbour offset -1 + a along a half axis, 0 along an integer one
            const int o0 = h[0] ? a - 1 : 0, o1 = h[1] ? b - 1 : 0, o2 = h[2] ? e - 1 : 0;
            const bool in = (o0 == 0 || ok[0]) && (o1 == 0 || ok[1]) && (o2 == 0 || ok[2]);
            acc += in ? F[o0 * st[0] + o1 * st[1] + o2 * st[2]] : T(0);
            cnt++;
          }
      dst[c * g.cs + p] = cnt == 4 ? T(0.25) * acc : cnt == 2 ? T(0.5) * acc : acc;
    }
  }
}

// ---------------------------------------------------------------------------
// particles
template <class T>
struct Parts3 {
  double* x; double* y; double* z;
  T* ux; T* uy; T* uz; T* w;
  uint32_t* id;
  int* fl;          // bit 0: alive
};


template <class T, int ORD>
__device__ __forceinline__ void shape_w(T t, T* w) {
  if (ORD == 3) weights3<T>(t, w);
  else weights1<T>(t, w);
}

// fields at a particle: each component from its own Yee position, the same shape along every axis
template <class T, int ORD>
__device__ void gather3(const G3& g, const T* const* fE, const T* const* fB, const double* pos, T* E, T* B,
                        bool nodal) {
  constexpr int NS = ORD == 3 ? 4 : 2;
  constexpr int SH = ORD == 3 ? 1 : 0;
  T w[3][2][NS];
  int b[3][2];
#pragma unroll
  for (int a = 0; a < 3; a++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const double X = pos[a] / g.d[a] - 0.5 * h;
      const double f = floor(X);
      shape_w<T, ORD>(T(X - f), w[a][h]);
      b[a][h] = (int)f - SH;
    }
#pragma unroll
  for (int c = 0; c < 6; c++) {
    const T* F = c < 3 ? fE[c] : fB[c - 3];
    // Yee locations, or the nodes for the 'momentum conserving' gather
    const int hx = nodal ? 0 : c < 3 ? (c == 0) : (c != 3), hy = nodal ? 0 : c < 3 ? (c == 1) : (c != 4),
              hz = nodal ? 0 : c < 3 ? (c == 2) : (c != 5);
    T acc = T(0);
    for (int l0 = 0; l0 < NS; l0++) {
      const T w0 = w[0][hx][l0];
      for (int l1 = 0; l1 < NS; l1++) {
        const T w01 = w0 * w[1][hy][l1];
        for (int l2 = 0; l2 < NS; l2++)
          acc += rd3(g, F, b[0][hx] + l0, b[1][hy] + l1, b[2][hz] + l2) * (w01 * w[2][hz][l2]);
      }
    }
    if (c < 3) E[c] = acc;
    else B[c - 3] = acc;
  }
}

// relativistic Boris push (textbook): u^{n-1/2} -> u^{n+1/2}, u = gamma v
template <class T>
__device__ __forceinline__ void boris3(T* u, const T* E, const T* B, T k) {
  const T ic2 = T(1.0 / (kC * kC));
  const T um0 = u[0] + k * E[0], um1 = u[1] + k * E[1], um2 = u[2] + k * E[2];
  const T gm = sqrt(T(1) + (um0 * um0 + um1 * um1 + um2 * um2) * ic2);
  const T kg = k / gm;   // one division each for k/gamma and 2/(1 + t^2)
  const T t0 = kg * B[0], t1 = kg * B[1], t2 = kg * B[2];
  const T tt = t0 * t0 + t1 * t1 + t2 * t2;
  const T sf = T(2) / (T(1) + tt);
  const T s0 = sf * t0, s1 = sf * t1, s2 = sf * t2;
  const T up0 = um0 + (um1 * t2 - um2 * t1), up1 = um1 + (um2 * t0 - um0 * t2), up2 = um2 + (um0 * t1 - um1 * t0);
  const T pl0 = um0 + (up1 * s2 - up2 * s1), pl1 = um1 + (up2 * s0 - up0 * s2), pl2 = um2 + (up0 * s1 - up1 * s0);
  u[0] = pl0 + k * E[0];
  u[1] = pl1 + k * E[1];
  u[2] = pl2 + k * E[2];
}

template <class T>
struct Fld3 {
  const T* fE[3];
  const T* fB[3];
  T* J[3];
};

// ---------------------------------------------------------------------------
// tiled push: particles sorted by tiles of TX x TY x TZ cells; one CTA per tile stages the six
// gather fields of the tile and its halo in shared memory, accumulates the current of its particles
// in a shared window with shared-memory atomics, and adds the window to J once
constexpr int TX = 4, TY = 4, TZ = 16;
// window nodes cell0-3 .. cell0+T+3: the gather and deposit stencils of a particle within half a cell of
// its tile (tile-local coordinate in [-1/2, T+1/2), which absorbs the rounding of the sort's cell index
// against the push's FP32 tile-local coordinate) moving less than one cell
constexpr int WM = 3;
constexpr int WX = TX + 2 * WM + 1, WY = TY + 2 * WM + 1, WZ = TZ + 2 * WM + 1;
constexpr int WN = WX * WY * WZ;
// window element stride along axis a
__host__ __device__ constexpr int wstride(int a) { return a == 0 ? WY * WZ : a == 1 ? WZ : 1; }
// The gathered fields need less: a cubic stencil of a particle within half a cell of its tile reaches
// nodes -2 .. T+2 (integer and half positions alike), so their window starts WGM = 2 before the tile
// and is T + 5 nodes long on each axis (the current window above keeps WM = 3 for the move). The
// smaller field window is what lets three CTAs share an SM.
constexpr int WGM = 2;
constexpr int WGX = TX + 2 * WGM + 1, WGY = TY + 2 * WGM + 1, WGZ = TZ + 2 * WGM + 1;
constexpr int WGN = WGX * WGY * WGZ;
// shared memory of the 3D push: the six gathered fields on the field window, the current on its window
template <class T>
constexpr int push3_smem() { return (int)((6 * WGN + 3 * WN) * sizeof(T)); }

struct Tiles3 {
  int nt[3];
  int* cnt;      // particles per tile (filled by the key pass)
  int* start;    // exclusive scan of cnt
  int* key;      // per particle: tile, -1 when dropped
  int* rank;     // per particle: rank inside its tile
};

__device__ __forceinline__ int tile_of(const G3& g, const Tiles3& t, const double* pos) {
  const int ci = (int)floor(pos[0] * g.id[0]), cj = (int)floor(pos[1] * g.id[1]), ck = (int)floor(pos[2] * g.id[2]);
  if (ci < 0 || cj < 0 || ck < 0 || ci >= g.n[0] || cj >= g.n[1] || ck >= g.n[2]) return -1;
  return ((ci / TX) * t.nt[1] + cj / TY) * t.nt[2] + ck / TZ;
}

// tile key and rank of every live particle (warp-aggregated counters); every slot below n (the host's
// bound on the count) gets a key, -1 beyond the device count, so that the scatter reads no stale key
template <class T>
__global__ void k3_tile_key(G3 g, Parts3<T> p, const Ctrl3* ctrl, Tiles3 t, int n) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = j < ctrl->count;
  int key = -1;
  if (in && (p.fl[j] & 1)) {
    const double pos[3] = {p.x[j], p.y[j], p.z[j]};
    key = tile_of(g, t, pos);
  }
  const unsigned act = __ballot_sync(0xffffffffu, key >= 0);
  if (key >= 0) {
    const unsigned grp = __match_any_sync(act, key);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(grp) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(t.cnt + key, __popc(grp));
    base = __shfl_sync(grp, base, leader);
    t.rank[j] = base + __popc(grp & ((1u << lane) - 1u));
  }
  if (j < n) t.key[j] = key;
}

// exclusive scan of the tile counts by one block, in chunks of 8192 counts staged with coalesced loads
// (each thread sums eight consecutive counts); the total becomes the particle count
__global__ void __launch_bounds__(1024) k3_scan_tiles(const int* cnt, int* start, int n, Ctrl3* ctrl) {
  constexpr int CH = 8192, PER = CH / 1024;
  __shared__ int buf[CH];
  __shared__ int part[1024];
  int carry = 0;
  for (int c0 = 0; c0 < n; c0 += CH) {
    for (int e = threadIdx.x; e < CH; e += 1024) buf[e] = c0 + e < n ? cnt[c0 + e] : 0;
    __syncthreads();
    int s = 0;
#pragma unroll
    for (int q = 0; q < PER; q++) s += buf[threadIdx.x * PER + q];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int v = threadIdx.x >= o ? part[threadIdx.x - o] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    int run = carry + part[threadIdx.x] - s;
#pragma unroll
    for (int q = 0; q < PER; q++) {
      const int v = buf[threadIdx.x * PER + q];
      buf[threadIdx.x * PER + q] = run;
      run += v;
    }
    const int tot = part[1023];
    __syncthreads();
    for (int e = threadIdx.x; e < CH; e += 1024)
      if (c0 + e < n) start[c0 + e] = buf[e];
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    start[n] = carry;
    ctrl->count = carry;
  }
}

template <class T>
__global__ void k3_tile_scatter(Parts3<T> src, Parts3<T> dst, Tiles3 t, int n_old) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n_old) return;
  const int key = t.key[j];
  if (key < 0) return;
  const int q = t.start[key] + t.rank[j];
  dst.x[q] = src.x[j]; dst.y[q] = src.y[j]; dst.z[q] = src.z[j];
  dst.ux[q] = src.ux[j]; dst.uy[q] = src.uy[j]; dst.uz[q] = src.uz[j];
  dst.w[q] = src.w[j]; dst.id[q] = src.id[j]; dst.fl[q] = 1;
}

template <class T, int ORD, bool MC>
__global__ void __launch_bounds__(256, 3) k3_push_tiles(G3 g, Fld3<T> f, Parts3<T> p, Tiles3 t, Ctrl3* ctrl, T kq,
                                                     Cq3<T> cq) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sF = reinterpret_cast<T*>(smraw);        // 6 x WGN gather fields
  T* sJ = sF + 6 * WGN;                       // 3 x WN current
  const int tile = blockIdx.x;
  const int p0 = t.start[tile], p1 = t.start[tile + 1];
  if (p1 <= p0) return;
  const int tz = tile % t.nt[2], r = tile / t.nt[2];
  const int ty = r % t.nt[1], tx = r / t.nt[1];
  const int c0[3] = {tx * TX, ty * TY, tz * TZ};          // the tile's first cell; the window starts WM before
  // the window line by line: a warp per (component, x, y) line, a lane per z node (WZ <= 32), so that the
  // index arithmetic is paid once per line; a window clear of the grid's faces skips the bounds checks
  static_assert(WZ <= 32, "one lane per z node of a window line");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const bool clear = c0[0] - WM >= 0 && c0[1] - WM >= 0 && c0[2] - WM >= 0 && c0[0] - WM + WX - 1 <= g.n[0] &&
                     c0[1] - WM + WY - 1 <= g.n[1] && c0[2] - WM + WZ - 1 <= g.n[2];
  const bool clear_g = c0[0] - WGM >= 0 && c0[1] - WGM >= 0 && c0[2] - WGM >= 0 &&
                       c0[0] - WGM + WGX - 1 <= g.n[0] && c0[1] - WGM + WGY - 1 <= g.n[1] &&
                       c0[2] - WGM + WGZ - 1 <= g.n[2];
  const long line_stride = (long)(g.n[1] + 1) * g.ldz;   // nid step along x
  // each warp takes SU consecutive lines at a time and issues their loads together (one round trip to
  // L2 or HBM per SU lines instead of one per line)
  static_assert(WGZ <= 32, "one lane per z node of a field-window line");
  constexpr int NL = 6 * WGX * WGY, SU = 8;
  for (int l0 = warp * SU; l0 < NL; l0 += nwarps * SU) {
    T v[SU];
#pragma unroll
    for (int u = 0; u < SU; u++) {
      const int line = l0 + u;
      v[u] = T(0);
      if (line < NL && lane < WGZ) {
        const int c = line / (WGX * WGY), ab = line - c * (WGX * WGY);
        const int a = ab / WGY, b = ab - a * WGY;
        const T* F =
            c == 0 ? f.fE[0] : c == 1 ? f.fE[1] : c == 2 ? f.fE[2] : c == 3 ? f.fB[0] : c == 4 ? f.fB[1] : f.fB[2];
        const int i = c0[0] - WGM + a, jj = c0[1] - WGM + b, k = c0[2] - WGM + lane;
        v[u] = clear_g ? F[(long)i * line_stride + (long)jj * g.ldz + k] : rd3(g, F, i, jj, k);
      }
    }
#pragma unroll
    for (int u = 0; u < SU; u++)
      if (l0 + u < NL && lane < WGZ) sF[(l0 + u) * WGZ + lane] = v[u];
  }
  for (int e = threadIdx.x; e < 3 * WN; e += blockDim.x) sJ[e] = T(0);
  __syncthreads();
  constexpr int NS = ORD == 3 ? 4 : 2;
  constexpr int SH = ORD == 3 ? 1 : 0;
  constexpr int W = NS + 1;
  // tile-local coordinates in cells: X = (pos - c0 d) / d; everything below runs in T (FP32 on the mixed
  // path: one FP64 subtraction and multiplication per axis to enter, one FP64 addition to leave)
  double org[3], inv[3];
  T dT[3], invT[3], lo[3], hi[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    org[a] = c0[a] * g.d[a];
    inv[a] = g.id[a];
    dT[a] = T(g.d[a]);
    invT[a] = T(inv[a]);
    lo[a] = T(g.lo[a] - c0[a]);
    hi[a] = T(g.hi[a] - c0[a] + (a == 2 ? 1 : 0));
  }
  const T dtT = T(g.dt);
  // J_q per unit weight: -q/(d_u d_v dt), from the host
  T cqw[3];
#pragma unroll
  for (int a = 0; a < 3; a++) cqw[a] = cq.v[a];
  for (int j = p0 + threadIdx.x; j < p1; j += blockDim.x) {
    const double pos[3] = {p.x[j], p.y[j], p.z[j]};
    T X[3];
    bool inside = true;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      X[a] = T((pos[a] - org[a]) * inv[a]);
      const int ext = a == 0 ? TX : a == 1 ? TY : TZ;
      if (!(X[a] >= T(-0.5)) || !(X[a] < T(ext) + T(0.5))) inside = false;
    }
    // the window covers the tile's cells and half a cell around them: a particle further out (never
    // expected after the sort) is left untouched and flagged
    if (!inside) {
      atomicOr(&ctrl->status, (int)ST_OUTSIDE);
      continue;
    }
    // gather from the staged window (field-window index = local cell + WGM)
    T wg[3][2][NS];
    int bl[3][2];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
      for (int h = 0; h < 2; h++) {
        const T Xs = X[a] - T(0.5) * T(h);
        const T fl = floor(Xs);
        shape_w<T, ORD>(Xs - fl, wg[a][h]);
        bl[a][h] = (int)fl - SH + WGM;
      }
    T EB[6];
#pragma unroll
    for (int c = 0; c < 6; c++) {
      // Yee locations; every component at the nodes for the 'momentum conserving' gather (MC). The
      // tensor-product sum taken axis by axis: z within each (x, y) row, then y, then x
      const int hx = MC ? 0 : c < 3 ? (c == 0) : (c != 3), hy = MC ? 0 : c < 3 ? (c == 1) : (c != 4),
                hz = MC ? 0 : c < 3 ? (c == 2) : (c != 5);
      const T* F = sF + c * WGN + (bl[0][hx] * WGY + bl[1][hy]) * WGZ + bl[2][hz];
      T acc = T(0);
#pragma unroll
      for (int l0 = 0; l0 < NS; l0++) {
        T accy = T(0);
#pragma unroll
        for (int l1 = 0; l1 < NS; l1++) {
          const T* row = F + (l0 * WGY + l1) * WGZ;
          T accz = T(0);
#pragma unroll
          for (int l2 = 0; l2 < NS; l2++) accz += row[l2] * wg[2][hz][l2];
          accy += wg[1][hy][l1] * accz;
        }
        acc += wg[0][hx][l0] * accy;
      }
      EB[c] = acc;
    }
    T u[3] = {p.ux[j], p.uy[j], p.uz[j]};
    boris3<T>(u, EB, EB + 3, kq);
    const T gm = sqrt(T(1) + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * T(1.0 / (kC * kC)));
    T X1[3], Dm[3];
    const T ig = T(1) / gm;
#pragma unroll
    for (int a = 0; a < 3; a++) {
      Dm[a] = dtT * (u[a] * ig);          // displacement [m]
      X1[a] = X[a] + Dm[a] * invT[a];
    }
    // Esirkepov into the shared window
    T S0[3][W], DS[3][W];
    int base[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      const T f0 = floor(X[a]), f1 = floor(X1[a]);
      base[a] = (int)(f0 < f1 ? f0 : f1) - SH;
      T wa[NS], wb[NS];
      shape_w<T, ORD>(X[a] - f0, wa);
      shape_w<T, ORD>(X1[a] - f1, wb);
      // each stencil starts at base or one cell above (moves below one cell): select with constant indices
      const bool up0 = f0 > f1, up1 = f1 > f0;
#pragma unroll
      for (int m = 0; m < W; m++) {
        const T s0 = up0 ? (m > 0 ? wa[m - 1] : T(0)) : (m < NS ? wa[m] : T(0));
        const T s1 = up1 ? (m > 0 ? wb[m - 1] : T(0)) : (m < NS ? wb[m] : T(0));
        S0[a][m] = s0;
        DS[a][m] = s1 - s0;
      }
      base[a] += WM;
    }
    // the prefix along q of W_q = DS_q tr(u, v) factorises: J_q(m_q, m_u, m_v) = cq tr(m_u, m_v) C_q(m_q),
    // C_q the running sum of DS_q; all loops unrolled so that the stencils stay in registers
    // C_q at the W - 1 edges between the stencil's nodes (its value past the last node is the total change
    // of the shape, zero)
    T Cm[3][W - 1];
#pragma unroll
    for (int a = 0; a < 3; a++) {
      T run = T(0);
#pragma unroll
      for (int m = 0; m < W - 1; m++) {
        run += DS[a][m];
        Cm[a][m] = run;
      }
    }
    const T wj = p.w[j];
    // the window offset of the stencil's first node; every term's offset from it is a compile-time
    // constant once the loops are unrolled
    const int off0 = (base[0] * WY + base[1]) * WZ + base[2];
#pragma unroll
    for (int q = 0; q < 3; q++) {
      const int u1 = (q + 1) % 3, v1 = (q + 2) % 3;
      bool moved = false;
#pragma unroll
      for (int m = 0; m < W; m++) moved |= DS[q][m] != T(0);
      if (!moved) continue;
      const T cq = cqw[q] * wj;
      T* Jq = sJ + q * WN + off0;
      // tr(u, v) = S0_u S0_v + DS_u S0_v / 2 + S0_u DS_v / 2 + DS_u DS_v / 3
      //          = S0_u (S0_v + DS_v / 2) + DS_u (S0_v / 2 + DS_v / 3), times cq
      T Av[W], Bv[W];
#pragma unroll
      for (int mv = 0; mv < W; mv++) {
        Av[mv] = cq * (S0[v1][mv] + T(0.5) * DS[v1][mv]);
        Bv[mv] = cq * (T(0.5) * S0[v1][mv] + DS[v1][mv] * T(1.0 / 3.0));
      }
#pragma unroll
      for (int mu = 0; mu < W; mu++)
#pragma unroll
        for (int mv = 0; mv < W; mv++) {
          const T ct = S0[u1][mu] * Av[mv] + DS[u1][mu] * Bv[mv];
          if (ct == T(0)) continue;
#pragma unroll
          for (int mq = 0; mq < W - 1; mq++) {
            const T v = ct * Cm[q][mq];
            if (v == T(0)) continue;
            atomicAdd(Jq + mq * wstride(q) + mu * wstride(u1) + mv * wstride(v1), v);
          }
        }
    }
    const double pn[3] = {pos[0] + (double)Dm[0], pos[1] + (double)Dm[1], pos[2] + (double)Dm[2]};
    p.x[j] = pn[0]; p.y[j] = pn[1]; p.z[j] = pn[2];
    p.ux[j] = u[0]; p.uy[j] = u[1]; p.uz[j] = u[2];
    bool out = false;
    if (sizeof(T) == 8) {
      // FP64 path: the removal decision on the physical position, as the method states it
#pragma unroll
      for (int a = 0; a < 3; a++) {
        const double lop = g.lo[a] * g.d[a];
        const double hip = g.hi[a] * g.d[a] + (a == 2 ? g.d[2] : 0.0);
        if (pn[a] < lop || pn[a] >= hip) out = true;
      }
    } else {
#pragma unroll
      for (int a = 0; a < 3; a++)
        if (X1[a] < lo[a] || X1[a] >= hi[a]) out = true;
    }
    if (out) p.fl[j] = 0;
  }
  __syncthreads();
  // the window's current added to J line by line, as it was staged
  for (int line = warp; line < 3 * WX * WY; line += nwarps) {
    if (lane >= WZ) continue;
    const T v = sJ[line * WZ + lane];
    if (v == T(0)) continue;
    const int c = line / (WX * WY), ab = line - c * (WX * WY);
    const int a = ab / WY, b = ab - a * WY;
    const int i = c0[0] - WM + a, jj = c0[1] - WM + b, kk = c0[2] - WM + lane;
    if (!clear && (i < 0 || i > g.n[0] || jj < 0 || jj > g.n[1] || kk < 0 || kk > g.n[2])) continue;
    T* J = c == 0 ? f.J[0] : c == 1 ? f.J[1] : f.J[2];
    atomicAdd(J + (long)i * line_stride + (long)jj * g.ldz + kk, v);
  }
}

// ---------------------------------------------------------------------------
// plasma: lattice rows, rigid ions as a separable column current
struct Lat3 {
  double h, gamma, beta, n0, z_start_lab, ramp_lab, length_lab;
  int ppc[3];
  int nxl, nyl;
};

__host__ __device__ inline double lab_density3(const Lat3& L, double zl) {
  if (zl < L.z_start_lab) return 0.0;
  const double r = zl - L.z_start_lab;
  if (L.ramp_lab > 0.0 && r < L.ramp_lab) return L.n0 * r / L.ramp_lab;
  const double plateau_end = L.ramp_lab + L.length_lab;
  if (L.length_lab > 0.0 && r >= plateau_end) return 0.0;
  return L.n0;
}

struct Rows8 {
  long long m[8];
  int n;
};

template <class T>
__global__ void k3_inject(G3 g, Parts3<T> p, const Ctrl3* ctrl, Lat3 L, Rows8 rows, double t) {
  const long per = (long)L.nxl * L.nyl;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= per * rows.n) return;
  const int r = (int)(e / per);
  const long ab = e - (long)r * per;
  const int a = (int)(ab / L.nyl), b = (int)(ab - (long)a * L.nyl);
  const long long m = rows.m[r];
  const double zlat = (m + 0.5) * L.h;
  const double n = L.gamma * lab_density3(L, L.gamma * zlat);
  const long q = (long)ctrl->count + e;
  p.x[q] = (g.lo[0] + (a + 0.5) / L.ppc[0]) * g.d[0];
  p.y[q] = (g.lo[1] + (b + 0.5) / L.ppc[1]) * g.d[1];
  p.z[q] = zlat - L.beta * kC * t;
  p.ux[q] = T(0);
  p.uy[q] = T(0);
  p.uz[q] = T(-L.gamma * L.beta * kC);
  p.w[q] = T(n * g.d[0] * g.d[1] * g.d[2] / (double)(L.ppc[0] * L.ppc[1] * L.ppc[2]));
  p.id[q] = (uint32_t)((unsigned long long)m * (unsigned long long)per + (unsigned long long)(a * (long)L.nyl + b));
  p.fl[q] = 1;
}

__global__ void k3_add_count(Ctrl3* c, int d) { c->count += d; }

// sum over n >= 0 of S(u + n): the prefix of the shape samples (Esirkepov's 1D flux)
__device__ __forceinline__ double cum_shape(int order, double u) {
  const double r = order == 3 ? 2.0 : 1.0;
  if (u >= r) return 0.0;
  if (u <= -r) return 1.0;
  double acc = 0.0;
  for (int n = 0; n < 5; n++) {
    const double s = fabs(u + n);
    double v = 0.0;
    if (order == 1) v = s < 1.0 ? 1.0 - s : 0.0;
    else if (s < 1.0) v = 2.0 / 3.0 - s * s + 0.5 * s * s * s;
    else if (s < 2.0) { const double t = 2.0 - s; v = t * t * t / 6.0; }
    acc += v;
  }
  return acc;
}

// Z(k) = sum over the live ion rows of w_m (C(Z1 - k) - C(Z0 - k)): the z-prefix of the rows' shape change.
// One warp per z node, its lanes over the rows near the node (strided), then a warp sum: the FP64 shape
// sums are latency-bound, so they are spread over many warps instead of run one node per thread.
__global__ void k3_ion_z(G3 g, Lat3 L, int order, long long mlo, long long mhi, double t0, double t1, double* Zs) {
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k > g.n[2]) return;   // warp-uniform
  const double dz = g.d[2], idz = g.id[2];
  const double vsh = L.beta * kC;
  long long m0 = (long long)floor(((k - 4) * dz + vsh * t0) / L.h - 0.5);
  long long m1 = (long long)ceil(((k + 4) * dz + vsh * t0) / L.h - 0.5);
  if (m0 < mlo) m0 = mlo;
  if (m1 > mhi - 1) m1 = mhi - 1;
  double acc = 0.0;
  for (long long m = m0 + lane; m <= m1; m += 32) {
    const double zl = (m + 0.5) * L.h;
    const double n = L.gamma * lab_density3(L, L.gamma * zl);
    if (n <= 0.0) continue;
    const double w = n * g.d[0] * g.d[1] * g.d[2] / (double)(L.ppc[0] * L.ppc[1] * L.ppc[2]);
    const double Z0 = (zl - vsh * t0) * idz, Z1 = (zl - vsh * t1) * idz;
    acc += w * (cum_shape(order, Z1 - k) - cum_shape(order, Z0 - k));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) Zs[k] = acc;
}

// J_z += coef Tx(i) Ty(j) Z(k), coef = -q_ion/(dx dy dt), on the nodes where T_x T_y is non-zero
// (i0 + blockIdx.z, j0 + blockIdx.y); KPT z nodes per thread, a block width apart
template <class T>
__global__ void __launch_bounds__(128) k3_ion_jz(G3 g, const double* Tx, const double* Ty, const double* Zs,
                                                 double coef, int i0, int j0, T* Jz) {
  const int i = i0 + blockIdx.z, j = j0 + blockIdx.y;
  const double f = coef * Tx[i] * Ty[j];
  if (f == 0.0) return;
  const int kb = blockIdx.x * 128 * KPT + threadIdx.x;
  // every load of the thread's KPT nodes issued before any store
  T jv[KPT];
  double zv[KPT];
#pragma unroll
  for (int kk = 0; kk < KPT; kk++) {
    const int k = min(kb + kk * 128, g.n[2]);
    zv[kk] = Zs[k];
    jv[kk] = Jz[nid(g, i, j, k)];
  }
#pragma unroll
  for (int kk = 0; kk < KPT; kk++) {
    const int k = kb + kk * 128;
    if (k > g.n[2]) break;
    const double v = f * zv[kk];
    if (v != 0.0) Jz[nid(g, i, j, k)] = jv[kk] + T(v);
  }
}

// charge density of the ion rows at time t: q/(dV) Tx(i) Ty(j) sum_m w_m S(Z_m - k)
__global__ void k3_ion_rho(G3 g, Lat3 L, int order, long long mlo, long long mhi, double t, const double* Tx,
                           const double* Ty, double* rho) {
  int i, j, k;
  if (!node_of(g, (long)blockIdx.x * blockDim.x + threadIdx.x, i, j, k)) return;
  if (Tx[i] == 0.0 || Ty[j] == 0.0) return;
  const double dz = g.d[2], vsh = L.beta * kC;
  long long m0 = (long long)floor(((k - 3) * dz + vsh * t) / L.h - 0.5);
  long long m1 = (long long)ceil(((k + 3) * dz + vsh * t) / L.h - 0.5);
  if (m0 < mlo) m0 = mlo;
  if (m1 > mhi - 1) m1 = mhi - 1;
  double acc = 0.0;
  for (long long m = m0; m <= m1; m++) {
    const double zl = (m + 0.5) * L.h;
    const double n = L.gamma * lab_density3(L, L.gamma * zl);
    if (n <= 0.0) continue;
    const double w = n * g.d[0] * g.d[1] * g.d[2] / (double)(L.ppc[0] * L.ppc[1] * L.ppc[2]);
    const double Z = (zl - vsh * t) / dz;
    const double s = fabs(Z - k);
    double v = 0.0;
    if (order == 1) v = s < 1.0 ? 1.0 - s : 0.0;
    else if (s < 1.0) v = 2.0 / 3.0 - s * s + 0.5 * s * s * s;
    else if (s < 2.0) { const double tt = 2.0 - s; v = tt * tt * tt / 6.0; }
    acc += w * v;
  }
  rho[nid(g, i, j, k)] += kQe * Tx[i] * Ty[j] * acc / (g.d[0] * g.d[1] * g.d[2]);
}

template <class T>
__global__ void k3_particle_rho(G3 g, Parts3<T> p, const Ctrl3* ctrl, int order, double q, double* rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ctrl->count || !(p.fl[j] & 1)) return;
  const double pos[3] = {p.x[j], p.y[j], p.z[j]};
  const double qw = q * (double)p.w[j] / (g.d[0] * g.d[1] * g.d[2]);
  double w[3][4];
  int b[3];
  const int NS = order == 3 ? 4 : 2, SH = order == 3 ? 1 : 0;
  for (int a = 0; a < 3; a++) {
    const double X = pos[a] / g.d[a], f = floor(X);
    if (order == 3) weights3<double>(X - f, w[a]);
    else weights1<double>(X - f, w[a]);
    b[a] = (int)f - SH;
  }
  for (int l0 = 0; l0 < NS; l0++)
    for (int l1 = 0; l1 < NS; l1++)
      for (int l2 = 0; l2 < NS; l2++) {
        const int i = b[0] + l0, jj = b[1] + l1, k = b[2] + l2;
        if (i < 0 || i > g.n[0] || jj < 0 || jj > g.n[1] || k < 0 || k > g.n[2]) continue;
        atomicAdd(rho + nid(g, i, jj, k), qw * w[0][l0] * w[1][l1] * w[2][l2]);
      }
}

// ---------------------------------------------------------------------------
// laser antenna: dual particle arrays (Sec. 3.1.2)
struct Ant3 {
  double x_center, y_center, w0, za;
  double D0, D1;     // displacement factors before and after the step (delta = G(x, y) D)
  double Q;          // charge of the moving partner
  int order;
};

template <class T>
__global__ void k3_antenna(G3 g, T* Jy, Ant3 a) {
  const int nyp = g.hi[1] - g.lo[1] + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (g.hi[0] - g.lo[0] + 1) * nyp) return;
  const int i = g.lo[0] + e / nyp, j = g.lo[1] + e % nyp;
  const double x = i * g.d[0], y = j * g.d[1];
  const double rx = x - a.x_center, ry = y - a.y_center;
  const double G = exp(-(rx * rx + ry * ry) / (a.w0 * a.w0));
  const double y0 = y + G * a.D0, y1 = y + G * a.D1;
  if (y0 == y1) return;
  const int NS = a.order == 3 ? 4 : 2, SH = a.order == 3 ? 1 : 0;
  double wx[4], wz[4], S0y[5], DSy[5];
  {
    const double X = x / g.d[0], fx = floor(X), Z = a.za / g.d[2], fz = floor(Z);
    if (a.order == 3) { weights3<double>(X - fx, wx); weights3<double>(Z - fz, wz); }
    else { weights1<double>(X - fx, wx); weights1<double>(Z - fz, wz); }
    const double A0 = y0 / g.d[1], A1 = y1 / g.d[1], f0 = floor(A0), f1 = floor(A1);
    const int by = (int)(f0 < f1 ? f0 : f1) - SH;
    double w0[4], w1[4];
    if (a.order == 3) { weights3<double>(A0 - f0, w0); weights3<double>(A1 - f1, w1); }
    else { weights1<double>(A0 - f0, w0); weights1<double>(A1 - f1, w1); }
    const int o0 = (int)f0 - SH - by, o1 = (int)f1 - SH - by;
    for (int m = 0; m <= NS; m++) {
      const double s0 = (m - o0 >= 0 && m - o0 < NS) ? w0[m - o0] : 0.0;
      const double s1 = (m - o1 >= 0 && m - o1 < NS) ? w1[m - o1] : 0.0;
      S0y[m] = s0;
      DSy[m] = s1 - s0;
    }
    const int bx = (int)fx - SH, bz = (int)fz - SH;
    // J_y(j+1/2) - J_y(j-1/2) = -Q/(dx dz dt) W_y, W_y = DS_y S0_z S0_x
    const double cy = -a.Q / (g.d[0] * g.d[2] * g.dt);
    for (int lz = 0; lz < NS; lz++)
      for (int lx = 0; lx < NS; lx++) {
        const double tr = wz[lz] * wx[lx];
        if (tr == 0.0) continue;
        double acc = 0.0;
        for (int m = 0; m <= NS; m++) {
          acc += cy * DSy[m] * tr;
          if (acc == 0.0) continue;
          const int ii = bx + lx, jj = by + m, kk = bz + lz;
          if (ii < 0 || ii > g.n[0] || jj < 0 || jj > g.n[1] || kk < 0 || kk > g.n[2]) continue;
          atomicAdd(Jy + nid(g, ii, jj, kk), T(acc));
        }
      }
  }
}

// charge of the antenna pairs (the moving partner +Q, its fixed twin -Q) added to rho
__global__ void k3_antenna_rho(G3 g, Ant3 a, double* rho) {
  const int nyp = g.hi[1] - g.lo[1] + 1;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (g.hi[0] - g.lo[0] + 1) * nyp) return;
  const int i = g.lo[0] + e / nyp, j = g.lo[1] + e % nyp;
  const double x = i * g.d[0], y = j * g.d[1];
  const double rx = x - a.x_center, ry = y - a.y_center;
  const double dl = exp(-(rx * rx + ry * ry) / (a.w0 * a.w0)) * a.D1;
  if (dl == 0.0) return;
  const int NS = a.order == 3 ? 4 : 2, SH = a.order == 3 ? 1 : 0;
  const double pos[2][3] = {{x, y + dl, a.za}, {x, y, a.za}};
  for (int s = 0; s < 2; s++) {
    const double q = (s == 0 ? a.Q : -a.Q) / (g.d[0] * g.d[1] * g.d[2]);
    double w[3][4];
    int b[3];
    for (int ax = 0; ax < 3; ax++) {
      const double X = pos[s][ax] / g.d[ax], f = floor(X);
      if (a.order == 3) weights3<double>(X - f, w[ax]);
      else weights1<double>(X - f, w[ax]);
      b[ax] = (int)f - SH;
    }
    for (int l0 = 0; l0 < NS; l0++)
      for (int l1 = 0; l1 < NS; l1++)
        for (int l2 = 0; l2 < NS; l2++) {
          const int ii = b[0] + l0, jj = b[1] + l1, kk = b[2] + l2;
          if (ii < 0 || ii > g.n[0] || jj < 0 || jj > g.n[1] || kk < 0 || kk > g.n[2]) continue;
          atomicAdd(rho + nid(g, ii, jj, kk), q * w[0][l0] * w[1][l1] * w[2][l2]);
        }
  }
}

// ---------------------------------------------------------------------------
// test beam (Sec. 3.1.1)
template <class T>
struct Beam3 {
  double *x, *y, *z;
  T *ux, *uy, *uz;
  double *tc, *zf0;
  T *uxb, *uyb, *uzb;
  int* fl;    // bit 0 alive, bit 1 active
  int n;
  T* w;       // self-consistent beam: macro-particle weights (self = 1)
  int self;
};

__global__ void k3_beam_vz(int n, const double* ux, const double* uy, const double* uz, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double gj = sqrt(1.0 + (ux[j] * ux[j] + uy[j] * uy[j] + uz[j] * uz[j]) / (kC * kC));
  atomicAdd(&acc[0], uz[j] / gj);
}

template <class T>
__global__ void k3_beam_transform(Beam3<T> b, const double* lx, const double* ly, const double* lz,
                                  const double* lux, const double* luy, const double* luz, double t_lab,
                                  double z_plane, double gam, double be, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  const double betab = acc[0] / b.n / kC;
  const double gj = sqrt(1.0 + (lux[j] * lux[j] + luy[j] * luy[j] + luz[j] * luz[j]) / (kC * kC));
  const double vx = lux[j] / gj, vy = luy[j] / gj, vz = luz[j] / gj;
  const double tcross = t_lab + (z_plane - lz[j]) / vz;
  b.x[j] = lx[j] + vx * (tcross - t_lab);
  b.y[j] = ly[j] + vy * (tcross - t_lab);
  const double tpc = gam * (tcross - be * z_plane / kC);
  const double zpc = gam * (z_plane - be * kC * tcross);
  const double den = 1.0 - be * betab;
  const double vxp = vx / (gam * den), vyp = vy / (gam * den), vzp = (vz - be * kC) / den;
  const double v2 = (vxp * vxp + vyp * vyp + vzp * vzp) / (kC * kC);
  const double gp = 1.0 / sqrt(1.0 - v2);
  b.uxb[j] = T(gp * vxp); b.uyb[j] = T(gp * vyp); b.uzb[j] = T(gp * vzp);
  b.ux[j] = b.uxb[j]; b.uy[j] = b.uyb[j]; b.uz[j] = b.uzb[j];
  b.tc[j] = tpc;
  b.zf0[j] = zpc;
  b.fl[j] = 1;
  atomicAdd(&acc[1], vzp);
}

template <class T>
__global__ void k3_beam_finish(Beam3<T> b, double t_now, double* acc) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  const double vbar = acc[1] / b.n;
  const double zf = b.zf0[j] - vbar * b.tc[j];
  b.zf0[j] = zf;
  b.z[j] = zf + vbar * t_now;
  if (j == 0) acc[2] = vbar;
}

__device__ __forceinline__ double bshape(int order, double s) {
  const double a = fabs(s);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { const double t = 2.0 - a; return t * t * t / 6.0; }
  return 0.0;
}

// Esirkepov current of one beam particle (charge * weight qw) moving p0 -> p1, added to J with global
// atomics (a beam has few particles): along axis q, J_q is the running sum over the q-nodes of
// -qw d_q / (dx dy dz dt) DS_q times the transverse weight S0u S0v + DSu S0v / 2 + S0u DSv / 2 + DSu DSv / 3
// (Esirkepov 2001), on a window of 9 nodes per axis starting 3 below the lower of the two cells
template <class T>
__device__ void beam_current3(const G3& g, T* const* J, int order, const double* p0, const double* p1, double qw) {
  constexpr int EW = 9;
  int base[3];
  double S0[3][EW], DS[3][EW];
  for (int a = 0; a < 3; a++) {
    const double A0 = p0[a] / g.d[a], A1 = p1[a] / g.d[a];
    base[a] = (int)floor(A0 < A1 ? A0 : A1) - 3;
    for (int m = 0; m < EW; m++) {
      S0[a][m] = bshape(order, A0 - (base[a] + m));
      DS[a][m] = bshape(order, A1 - (base[a] + m)) - S0[a][m];
    }
  }
  for (int q = 0; q < 3; q++) {
    const int u = (q + 1) % 3, v = (q + 2) % 3;
    const double cq = -qw * g.d[q] / (g.d[0] * g.d[1] * g.d[2] * g.dt);
    for (int mu = 0; mu < EW; mu++)
      for (int mv = 0; mv < EW; mv++) {
        const double tr = S0[u][mu] * S0[v][mv] + 0.5 * DS[u][mu] * S0[v][mv] + 0.5 * S0[u][mu] * DS[v][mv] +
                          DS[u][mu] * DS[v][mv] / 3.0;
        if (tr == 0.0) continue;
        double acc = 0.0;
        for (int mq = 0; mq < EW; mq++) {
          acc += cq * DS[q][mq] * tr;
          if (acc == 0.0) continue;
          int idx[3];
          idx[q] = base[q] + mq; idx[u] = base[u] + mu; idx[v] = base[v] + mv;
          if (idx[0] < 0 || idx[0] > g.n[0] || idx[1] < 0 || idx[1] > g.n[1] || idx[2] < 0 || idx[2] > g.n[2]) continue;
          atomicAdd(J[q] + nid(g, idx[0], idx[1], idx[2]), T(acc));
        }
      }
  }
}

template <class T, int ORD>
__global__ void k3_beam_push(G3 g, Fld3<T> f, Beam3<T> b, double tn, double tn1, const double* acc, T kq,
                             int nodal) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n) return;
  int fl = b.fl[j];
  if (!(fl & 1)) return;
  double lo[3], hi[3];
  for (int a = 0; a < 3; a++) { lo[a] = g.lo[a] * g.d[a]; hi[a] = g.hi[a] * g.d[a]; }
  hi[2] += g.d[2];
  if (!(fl & 2)) {
    if (tn >= b.tc[j]) {
      fl |= 2;
      b.ux[j] = b.uxb[j]; b.uy[j] = b.uyb[j]; b.uz[j] = b.uzb[j];
      const double q[3] = {b.x[j], b.y[j], b.z[j]};
      for (int a = 0; a < 3; a++)
        if (q[a] < lo[a] || q[a] >= hi[a]) fl &= ~1;
      b.fl[j] = fl;
      if (!(fl & 1)) return;
    } else {
      const double zn = b.zf0[j] + acc[2] * tn1;
      // self-consistent beam: a frozen particle inside the particle domain carries its charge along z
      if (b.self) {
        const double p0[3] = {b.x[j], b.y[j], b.z[j]}, p1[3] = {b.x[j], b.y[j], zn};
        bool in = zn >= lo[2] && zn < hi[2];
        for (int a = 0; a < 3; a++) in = in && p0[a] >= lo[a] && p0[a] < hi[a];
        if (in) beam_current3<T>(g, f.J, ORD, p0, p1, -kQe * (double)b.w[j]);
      }
      b.z[j] = zn;
      return;
    }
  }
  const double pos[3] = {b.x[j], b.y[j], b.z[j]};
  T E[3], B[3];
  gather3<T, ORD>(g, f.fE, f.fB, pos, E, B, nodal != 0);
  T u[3] = {b.ux[j], b.uy[j], b.uz[j]};
  boris3<T>(u, E, B, kq);
  const T gm = sqrt(T(1) + (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * T(1.0 / (kC * kC)));
  double pn[3];
  for (int a = 0; a < 3; a++) pn[a] = pos[a] + g.dt * (double)(u[a] / gm);
  if (b.self) beam_current3<T>(g, f.J, ORD, pos, pn, -kQe * (double)b.w[j]);
  b.x[j] = pn[0]; b.y[j] = pn[1]; b.z[j] = pn[2];
  b.ux[j] = u[0]; b.uy[j] = u[1]; b.uz[j] = u[2];
  for (int a = 0; a < 3; a++)
    if (pn[a] < lo[a] || pn[a] >= hi[a]) fl &= ~1;
  b.fl[j] = fl;
}

// ---------------------------------------------------------------------------
// Self-field of the frozen beam in 3D (Sec. 3.1.1, PR-27): d2phi/dx2 + d2phi/dy2 + d2phi/dz2 / gamma_v^2 =
// -rho/eps0 with phi = 0 on the PEC walls, in the Yee mesh's second differences, solved by sine transforms
// (DST-I) along the three axes; E = -grad phi with E_z divided by gamma_v^2, B = v z x E / c^2 (B_x = -v E_y
// / c^2, B_y = v E_x / c^2) at their Yee positions. The solve works on an unpadded (nx+1)(ny+1)(nz+1) array
// (z fastest), FP64 throughout; a one-time set-up.

// charge density of the frozen beam particles inside the particle domain, positions `shift` seconds on
template <class T>
__global__ void k3_beam_rho(G3 g, Beam3<T> b, int order, double shift, const double* acc, double* rho) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b.n || (b.fl[j] & 3) != 1) return;
  const double r[3] = {b.x[j], b.y[j], b.z[j] + acc[2] * shift};
  for (int a = 0; a < 3; a++) {
    const double lo = g.lo[a] * g.d[a], hi = (g.hi[a] + (a == 2 ? 1 : 0)) * g.d[a];
    if (!(r[a] >= lo && r[a] < hi)) return;
  }
  const double qw = -kQe * (double)b.w[j] / (g.d[0] * g.d[1] * g.d[2]);
  int f[3];
  for (int a = 0; a < 3; a++) f[a] = (int)floor(r[a] / g.d[a]);
  const long L = g.n[2] + 1, PL = (long)(g.n[1] + 1) * L;
  for (int i = f[0] - 2; i <= f[0] + 3; i++) {
    const double wx = bshape(order, r[0] / g.d[0] - i);
    if (wx == 0.0 || i < 0 || i > g.n[0]) continue;
    for (int jj = f[1] - 2; jj <= f[1] + 3; jj++) {
      const double wy = bshape(order, r[1] / g.d[1] - jj);
      if (wy == 0.0 || jj < 0 || jj > g.n[1]) continue;
      for (int k = f[2] - 2; k <= f[2] + 3; k++) {
        const double wz = bshape(order, r[2] / g.d[2] - k);
        if (wz == 0.0 || k < 0 || k > g.n[2]) continue;
        atomicAdd(rho + i * PL + jj * L + k, qw * wx * wy * wz);
      }
    }
  }
}

// out(a, b, m) = 2 sum_{j=1}^{N-1} in(a, b, j) sin(pi j m / N), m = 1..N-1, for the interior outer indices
// a = 1..na-2, b = 1..nb-2 (strides sa, sb; the transform index stride si); tab[t] = sin(pi t / N), t < 2N.
// Threads run over m when si == 1 (the inputs of a row are shared), else over b (stride 1: coalesced).
__global__ void k3_dst(const double* in, double* out, const double* tab, int N, int na, int nb, long sa, long sb,
                       long si) {
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long cm = N - 1, ca = na - 2, cb = nb - 2;
  if (id >= cm * ca * cb) return;
  long a, b, m;
  if (si == 1) { m = 1 + id % cm; const long r = id / cm; b = 1 + r % cb; a = 1 + r / cb; }
  else { b = 1 + id % cb; const long r = id / cb; a = 1 + r % ca; m = 1 + r / ca; }
  const double* src = in + a * sa + b * sb;
  const int twoN = 2 * N;
  int t = 0;
  double acc = 0.0;
  for (int jj = 1; jj < N; jj++) {
    t += (int)m;
    if (t >= twoN) t -= twoN;
    acc += src[(long)jj * si] * tab[t];
  }
  out[a * sa + b * sb + m * si] = 2.0 * acc;
}

__global__ void k3_poisson_divide(double* ph, G3 g, double gv2) {
  const long L = g.n[2] + 1, PL = (long)(g.n[1] + 1) * L;
  const long cz = g.n[2] - 1, cy = g.n[1] - 1, cx = g.n[0] - 1;
  const long id = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= cx * cy * cz) return;
  const int k = 1 + (int)(id % cz), j = 1 + (int)((id / cz) % cy), i = 1 + (int)(id / (cz * cy));
  const double lx = -(2.0 - 2.0 * cospi((double)i / g.n[0])) / (g.d[0] * g.d[0]);
  const double ly = -(2.0 - 2.0 * cospi((double)j / g.n[1])) / (g.d[1] * g.d[1]);
  const double lz = -(2.0 - 2.0 * cospi((double)k / g.n[2])) / (g.d[2] * g.d[2]);
  const long p = i * PL + j * L + k;
  // each inverse DST-I is the forward one over 2N
  ph[p] = -ph[p] / kEps0 / (lx + ly + lz / gv2) / (8.0 * g.n[0] * g.n[1] * g.n[2]);
}

// phi = 0 on the six faces of the box (the transforms leave the deposited density there)
__global__ void k3_zero_faces(double* ph, G3 g) {
  const long L = g.n[2] + 1, PL = (long)(g.n[1] + 1) * L;
  const long n = PL * (g.n[0] + 1);
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const int k = (int)(e % L), j = (int)((e / L) % (g.n[1] + 1)), i = (int)(e / PL);
  if (i == 0 || i == g.n[0] || j == 0 || j == g.n[1] || k == 0 || k == g.n[2]) ph[e] = 0.0;
}

// mode 0: E_x, E_y, E_z added to E; mode 1: B_x, B_y added to B (from the earlier positions)
template <class T>
__global__ void k3_self_field_add(G3 g, T* E, T* B, const double* ph, double gv2, const double* acc, int mode) {
  const long L = g.n[2] + 1, PL = (long)(g.n[1] + 1) * L;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= PL * (g.n[0] + 1)) return;
  const int k = (int)(e % L), j = (int)((e / L) % (g.n[1] + 1)), i = (int)(e / PL);
  const long q = nid(g, i, j, k);
  if (mode == 0) {
    if (i < g.n[0]) E[q] += T(-(ph[e + PL] - ph[e]) / g.d[0]);
    if (j < g.n[1]) E[g.cs + q] += T(-(ph[e + L] - ph[e]) / g.d[1]);
    if (k < g.n[2]) E[2 * g.cs + q] += T(-(ph[e + 1] - ph[e]) / g.d[2] / gv2);
  } else {
    const double f = acc[2] / (kC * kC);
    if (j < g.n[1] && k < g.n[2]) {
      const double ey0 = -(ph[e + L] - ph[e]) / g.d[1], ey1 = -(ph[e + L + 1] - ph[e + 1]) / g.d[1];
      B[q] += T(-f * 0.5 * (ey0 + ey1));
    }
    if (i < g.n[0] && k < g.n[2]) {
      const double ex0 = -(ph[e + PL] - ph[e]) / g.d[0], ex1 = -(ph[e + PL + 1] - ph[e + 1]) / g.d[0];
      B[g.cs + q] += T(f * 0.5 * (ex0 + ex1));
    }
  }
}

// ---------------------------------------------------------------------------
// lab-frame samples (Sec. 3.2, PR-16): one transverse slice per row
template <class T>
__device__ __forceinline__ double interp_z3(const G3& g, const T* F, int i, int j, double zp, double stz) {
  const double Z = zp / g.d[2] - stz;
  const double kf = floor(Z);
  const int k = (int)kf;
  const double f = Z - kf;
  return (1.0 - f) * (double)rd3(g, F, i, j, k) + f * (double)rd3(g, F, i, j, k + 1);
}

template <class T>
__global__ void k3_btd(G3 g, const T* E, const T* B, T* out, int which, double wgt, double zp, double gam, double be) {
  const int nyp = g.n[1] + 1;
  const long plane = (long)(g.n[0] + 1) * nyp;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= plane) return;
  const int i = (int)(e / nyp), j = (int)(e - (long)i * nyp);
  if (which == 0) {
    const double ex = interp_z3(g, E, i, j, zp, 0.0);
    const double ey = interp_z3(g, E + g.cs, i, j, zp, 0.0);
    const double ez = interp_z3(g, E + 2 * g.cs, i, j, zp, 0.5);
    out[0 * plane + e] += T(wgt * gam * ex);
    out[1 * plane + e] += T(wgt * gam * ey);
    out[2 * plane + e] += T(wgt * ez);
    out[3 * plane + e] += T(wgt * (-gam * be * ey / kC));
    out[4 * plane + e] += T(wgt * (gam * be * ex / kC));
  } else {
    const double bx = interp_z3(g, B, i, j, zp, 0.5);
    const double by = interp_z3(g, B + g.cs, i, j, zp, 0.5);
    const double bz = interp_z3(g, B + 2 * g.cs, i, j, zp, 0.0);
    out[0 * plane + e] += T(wgt * gam * be * kC * by);
    out[1 * plane + e] += T(wgt * (-gam * be * kC * bx));
    out[3 * plane + e] += T(wgt * gam * bx);
    out[4 * plane + e] += T(wgt * gam * by);
    out[5 * plane + e] += T(wgt * bz);
  }
}

// ---------------------------------------------------------------------------
// diagnostics: out [0] n_e, [1] n_beam_active, [2] sum gamma_lab, [3] sum gamma_lab^2, [4] field energy,
// [5] weight of the electrons above the trapping threshold
template <class T>
__global__ void k3_stats(G3 g, const T* E, const T* B, Parts3<T> p, const Ctrl3* ctrl, Beam3<T> b, double gam,
                         double be, double trap, double* out) {
  __shared__ double red[6][256];
  const long tid = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const long nthr = (long)gridDim.x * blockDim.x;
  double v[6] = {0, 0, 0, 0, 0, 0};
  const long n = ctrl->count;
  if (sizeof(T) == 4) {
    // FP32 momenta: the lab-gamma test and the per-thread sums in FP32, loads issued without a branch
    const float ic2 = float(1.0 / (kC * kC)), ic = float(1.0 / kC);
    const float gamf = float(gam), bef = float(be), trapf = float(trap);
    int ne = 0;
    float wt = 0.f;
#pragma unroll 4
    for (long j = tid; j < n; j += nthr) {
      const bool live = (p.fl[j] & 1) != 0;
      ne += live ? 1 : 0;
      if (trap > 0.0) {
        const float ux = float(p.ux[j]), uy = float(p.uy[j]), uz = float(p.uz[j]), w = float(p.w[j]);
        const float gp = sqrtf(1.f + (ux * ux + uy * uy + uz * uz) * ic2);
        if (live && gamf * (gp + bef * uz * ic) > trapf) wt += w;
      }
    }
    v[0] = ne;
    v[5] = wt;
  } else {
    for (long j = tid; j < n; j += nthr) {
      if (!(p.fl[j] & 1)) continue;
      v[0] += 1.0;
      if (trap > 0.0) {
        const double ux = p.ux[j], uy = p.uy[j], uz = p.uz[j];
        const double gp = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
        if (gam * (gp + be * uz / kC) > trap) v[5] += (double)p.w[j];
      }
    }
  }
  for (long j = tid; j < b.n; j += nthr) {
    if ((b.fl[j] & 3) != 3) continue;
    const double ux = b.ux[j], uy = b.uy[j], uz = b.uz[j];
    const double gp = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) / (kC * kC));
    const double gl = gam * (gp + be * uz / kC);
    v[1] += 1; v[2] += gl; v[3] += gl * gl;
  }
  const double dV = g.d[0] * g.d[1] * g.d[2];
  if (sizeof(T) == 4) {
    // FP32 fields: each thread sums its nodes' energy density in FP32 (a few hundred terms), the blocks
    // and the grid reduce in FP64 (the FP64 pipe of this GPU is narrow)
    T acc = T(0);
#pragma unroll 4
    for (long q = tid; q < g.cs; q += nthr) {
      const T e2 = E[q] * E[q] + E[g.cs + q] * E[g.cs + q] + E[2 * g.cs + q] * E[2 * g.cs + q];
      const T b2 = B[q] * B[q] + B[g.cs + q] * B[g.cs + q] + B[2 * g.cs + q] * B[2 * g.cs + q];
      acc += T(kEps0) * e2 + b2 * T(kEps0 * kC * kC);
    }
    v[4] = 0.5 * (double)acc * dV;
  } else {
    for (long q = tid; q < g.cs; q += nthr) {
      const double e2 =
          (double)E[q] * E[q] + (double)E[g.cs + q] * E[g.cs + q] + (double)E[2 * g.cs + q] * E[2 * g.cs + q];
      const double b2 =
          (double)B[q] * B[q] + (double)B[g.cs + q] * B[g.cs + q] + (double)B[2 * g.cs + q] * B[2 * g.cs + q];
      v[4] += 0.5 * (kEps0 * e2 + b2 * (kEps0 * kC * kC)) * dV;
    }
  }
  for (int c = 0; c < 6; c++) red[c][threadIdx.x] = v[c];
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o)
      for (int c = 0; c < 6; c++) red[c][threadIdx.x] += red[c][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 6; c++) atomicAdd(out + c, red[c][0]);
}

// ---------------------------------------------------------------------------
// compaction of the live particles into the other buffer set
__global__ void k3_live_per_block(const int* fl, const Ctrl3* ctrl, int* bc) {
  __shared__ int s;
  if (threadIdx.x == 0) s = 0;
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int live = (j < ctrl->count && (fl[j] & 1)) ? 1 : 0;
  const int wsum = __popc(__ballot_sync(0xffffffffu, live));
  if ((threadIdx.x & 31) == 0 && wsum) atomicAdd(&s, wsum);
  __syncthreads();
  if (threadIdx.x == 0) bc[blockIdx.x] = s;
}

// exclusive scan of nb block counts by one block of 1024 threads; the total becomes the new count
__global__ void __launch_bounds__(1024) k3_scan_blocks(int* bc, int nb, Ctrl3* ctrl) {
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
__global__ void k3_scatter(Parts3<T> src, Parts3<T> dst, const int* bo, int n_old) {
  __shared__ int wo[8];
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int live = (j < n_old && (src.fl[j] & 1)) ? 1 : 0;
  const unsigned m = __ballot_sync(0xffffffffu, live);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) wo[wid] = __popc(m);
  __syncthreads();
  int off = bo[blockIdx.x];
  for (int w = 0; w < wid; w++) off += wo[w];
  if (!live) return;
  const int q = off + __popc(m & ((1u << lane) - 1u));
  dst.x[q] = src.x[j]; dst.y[q] = src.y[j]; dst.z[q] = src.z[j];
  dst.ux[q] = src.ux[j]; dst.uy[q] = src.uy[j]; dst.uz[q] = src.uz[j];
  dst.w[q] = src.w[j]; dst.id[q] = src.id[j]; dst.fl[q] = 1;
}

// ---------------------------------------------------------------------------
template <class T>
__global__ void k3_out_field(G3 g, const T* F, double* dst) {
  int i, j, k;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!node_of(g, e, i, j, k)) return;
  dst[e] = (double)F[nid(g, i, j, k)];
}

template <class T>
__global__ void k3_in_field(G3 g, const double* src, T* F) {
  int i, j, k;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!node_of(g, e, i, j, k)) return;
  F[nid(g, i, j, k)] = T(src[e]);
}

__global__ void k3_out_rho(G3 g, const double* rho, double* dst) {
  int i, j, k;
  const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (!node_of(g, e, i, j, k)) return;
  dst[e] = rho[nid(g, i, j, k)];
}

// ---------------------------------------------------------------------------
double cfl3(double a, double b, double gg, double dx, double dy, double dz, double theta) {
  const double kx = 1.0 / (dx * dx), ky = 1.0 / (dy * dy), kz = 1.0 / (dz * dz);
  double m = std::min(dx, std::min(dy, dz));
  const double pair = std::max(kx + ky, std::max(kx + kz, ky + kz));
  const double t1 = (a - 4.0 * gg) * pair, t2 = (a - 4.0 * b + 4.0 * gg) * (kx + ky + kz);
  if (t1 > 0 && 1.0 / std::sqrt(t1) < m) m = 1.0 / std::sqrt(t1);
  if (t2 > 0 && 1.0 / std::sqrt(t2) < m) m = 1.0 / std::sqrt(t2);
  return m / kC * std::sqrt((2.0 + theta) / (2.0 + 3.0 * theta));
}

double host_sigma(const pic_config& c, double pos, int n, double d_cell) {
  const int L = c.pml_cells;
  if (L <= 0) return 0.0;
  double d = 0.0;
  if (pos < L) d = L - pos;
  if (pos > n - L) d = pos - (n - L);
  if (d <= 0.0) return 0.0;
  return c.pml_sigma_max * kC / d_cell * std::pow(d / c.pml_delta, c.pml_power);
}

double shape_h(int order, double s) {
  const double a = std::fabs(s);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { const double t = 2.0 - a; return t * t * t / 6.0; }
  return 0.0;
}


template <class T>
struct Sim3 : Sim3Api {
  pic_config cfg;
  G3 g;
  cudaStream_t s;
  pic_alloc_fn alloc;
  pic_free_fn freef;
  void* user;
  std::vector<std::pair<void*, size_t>> allocs;
  std::string err;
  int st = PIC_OK;
  int64_t nl = 0;
  double gamma = 1, beta = 0;
  long step = 0;
  // fields (3-component blocks)
  T *E = nullptr, *B = nullptr, *J = nullptr, *Ep = nullptr, *Eb = nullptr;
  T *Es = nullptr, *Bs = nullptr;     // 6 split parts each
  T *fE = nullptr, *fB = nullptr, *tmp = nullptr, *tmp2 = nullptr;
  double* rho = nullptr;              // scratch for PIC_RHO
  double* out_d = nullptr;            // copy-out scratch
  Pml3<T> pm;
  Taps3<T> taps;
  // the fused x-y filter: tensor maps of the blocks it reads (gather copies and current), when it applies
  bool xy_ok = false;
  CUtensorMap xy_map[3];
  const T* xy_base[3] = {nullptr, nullptr, nullptr};
  Cq3<T> cq_e;
  bool nodal = false;     // 'momentum conserving' gather (pic_config.gather_scheme = 1)
  T* nF = nullptr;        // its node values: Ex, Ey, Ez, Bx, By, Bz
  int P = 0;
  // particles
  Parts3<T> P2[2];
  int cur = 0;
  long cap = 0, count_ub = 0;
  Ctrl3* ctrl = nullptr;
  int* blk = nullptr;
  long blk_cap = 0;
  int64_t compactions = 0;
  Tiles3 tl{};
  int ntiles = 0;
  long key_cap = 0;
  // plasma
  bool loaded = false;
  Lat3 lat;
  long long row_next = 0, mlo = 0;
  double* Tx = nullptr;
  double* Ty = nullptr;
  double* Zs = nullptr;
  int ion_i0 = 0, ion_i1 = 0, ion_j0 = 0, ion_j1 = 0;   // node range where T_x, T_y are non-zero
  bool ions = false;
  // laser
  bool has_laser = false;
  pic_laser las;
  double E0 = 0, Qpair = 0, Dn = 0;
  // beam
  Beam3<T> bm{};
  bool has_beam = false;
  double* bacc = nullptr;
  double* sred = nullptr;
  // lab samples
  std::vector<double> rz, rt;
  std::vector<int> rdone;
  T* rout = nullptr;
  // timing
  bool timing_on = false;
  int timing_which = 0;   // 0: the push kernel; 1: the field kernels (Faraday, Friedman, filters, Ampere)
  double t_ms = 0;
  std::vector<cudaEvent_t> tev;
  int64_t t_n = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;

  ~Sim3() override {
    if (s) cudaStreamSynchronize(s);
    for (auto& a : allocs) {
      if (freef) freef(a.first, a.second, (void*)s, user);
      else cudaFree(a.first);
    }
    for (auto e : tev) cudaEventDestroy(e);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
  }

  int fail(int code, const std::string& m) {
    if (st == PIC_OK) { st = code; err = m; }
    return code;
  }

  template <class X>
  X* dal(size_t n) {
    size_t bytes = (n * sizeof(X) + 255) & ~size_t(255);
    if (!bytes) bytes = 256;
    void* p = nullptr;
    if (alloc) p = alloc(bytes, (void*)s, user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) return nullptr;
    allocs.emplace_back(p, bytes);
    cudaMemsetAsync(p, 0, bytes, s);
    return (X*)p;
  }

  void dfree(void* p) {
    for (size_t i = 0; i < allocs.size(); i++)
      if (allocs[i].first == p) {
        cudaStreamSynchronize(s);
        if (freef) freef(p, allocs[i].second, (void*)s, user);
        else cudaFree(p);
        allocs.erase(allocs.begin() + i);
        return;
      }
  }

  long nodes() const { return (long)(g.n[0] + 1) * (g.n[1] + 1) * (g.n[2] + 1); }

  int init(const pic_config* c) {
    cfg = *c;
    gamma = c->gamma_boost < 1.0 ? 1.0 : c->gamma_boost;
    beta = std::sqrt(1.0 - 1.0 / (gamma * gamma));
    g.n[0] = c->nx; g.n[1] = c->ny; g.n[2] = c->nz;
    g.d[0] = c->dx; g.d[1] = c->dy; g.d[2] = (1.0 + beta) * gamma * c->dz_lab;   // Sec. 5.1.1
    for (int a = 0; a < 3; a++) g.id[a] = 1.0 / g.d[a];
    const double dt_cfl = cfl3(c->ck_alpha, c->ck_beta, c->ck_gamma, g.d[0], g.d[1], g.d[2], c->theta);
    g.dt = c->dt > 0.0 ? c->dt : c->courant * dt_cfl;
    const double vol_dt = g.d[0] * g.d[1] * g.d[2] * g.dt;
    for (int a = 0; a < 3; a++) cq_e.v[a] = T(kQe * g.d[a] / vol_dt);   // -q d_a/(d_x d_y d_z dt), q = -e
    if (!(g.dt > 0.0)) return fail(PIC_EINVAL, "dt <= 0");
    if (g.dt > dt_cfl * (1.0 + 1e-12)) return fail(PIC_ECFL, "dt above the 3D stability limit");
    P = c->filter_passes + (c->filter_compensate ? 1 : 0);
    FilterSpec fs{};
    fs.passes = c->filter_passes; fs.stride = c->filter_stride; fs.compensate = c->filter_compensate;
    for (int q = 0; q < 4; q++) fs.strides[q] = c->filter_stride_set[q];
    const int H = filter_halo(fs);
    if (H > FILTER_HMAX) return fail(PIC_EINVAL, "filter halo too wide");
    const int guard = c->particle_guard >= 0 ? c->particle_guard : (c->shape_order == 3 ? 3 : 2) + H + 2;
    if (guard < (c->shape_order == 3 ? 3 : 2) + H + 1) return fail(PIC_EINVAL, "particle guard too small");
    for (int a = 0; a < 3; a++) {
      g.lo[a] = c->pml_cells + guard;
      g.hi[a] = g.n[a] - c->pml_cells - guard;
      if (g.hi[a] - g.lo[a] < 2 || g.lo[a] < 4) return fail(PIC_EINVAL, "3D box too small for the PML and guard");
    }
    const int align = 128 / (int)sizeof(T);
    g.ldz = ((c->nz + 1 + align - 1) / align) * align;
    g.cs = (long)(c->nx + 1) * (c->ny + 1) * g.ldz;
    const size_t cs = (size_t)g.cs;
    E = dal<T>(3 * cs); B = dal<T>(3 * cs); J = dal<T>(3 * cs); Ep = dal<T>(3 * cs); Eb = dal<T>(3 * cs);
    nodal = c->gather_scheme == 1;
    if (nodal) {
      nF = dal<T>(6 * cs);
      if (!nF) return fail(PIC_ENOMEM, "allocation failed");
    }
    fE = dal<T>(3 * cs); fB = dal<T>(3 * cs); tmp = dal<T>(cs); tmp2 = dal<T>(cs);
    Es = dal<T>(6 * cs); Bs = dal<T>(6 * cs);
    ctrl = dal<Ctrl3>(1);
    bacc = dal<double>(8);
    sred = dal<double>(8);
    if (!E || !B || !J || !Ep || !Eb || !fE || !fB || !tmp || !tmp2 || !Es || !Bs || !ctrl || !bacc || !sred)
      return fail(PIC_ENOMEM, "allocation failed");
    // PML tables per axis, integer and half positions
    for (int a = 0; a < 3; a++) {
      const int n = g.n[a];
      std::vector<T> sgv(n + 2), xiv(n + 2), cfv(n + 2);
      for (int h = 0; h < 2; h++) {
        for (int i = 0; i <= n + 1; i++) {
          const double sg = i <= n ? host_sigma(cfg, i + 0.5 * h, n, g.d[a]) : 0.0;
          const double xi = c->pml_xi_exp ? std::exp(-sg * g.dt) : (1.0 - 0.5 * sg * g.dt) / (1.0 + 0.5 * sg * g.dt);
          sgv[i] = T(sg);
          xiv[i] = T(xi);
          cfv[i] = T(sg > 0.0 ? (1.0 - xi) / sg : g.dt);
        }
        T* d_s = dal<T>(n + 2);
        T* d_x = dal<T>(n + 2);
        T* d_c = dal<T>(n + 2);
        if (!d_s || !d_x || !d_c) return fail(PIC_ENOMEM, "allocation failed");
        cudaMemcpyAsync(d_s, sgv.data(), sizeof(T) * (n + 2), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_x, xiv.data(), sizeof(T) * (n + 2), cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_c, cfv.data(), sizeof(T) * (n + 2), cudaMemcpyHostToDevice, s);
        cudaStreamSynchronize(s);
        pm.sg[a][h] = d_s; pm.xi[a][h] = d_x; pm.cf[a][h] = d_c;
        pm.id[a] = T(g.id[a]);
      }
    }
    // composed filter taps along one axis: P passes of (1-a)/2, a, (1-a)/2 at stride s; a wide-band filter
    // (the passes repeated at each stride of a set) is composed densely over offsets -H..H (stride 1)
    const bool wide = fs.strides[0] > 0;
    const int R = wide ? H : P;
    std::vector<double> t(2 * R + 1, 0.0);
    t[R] = 1.0;
    for (int q = 0; q < (wide ? 4 : 1); q++) {
      const int st = wide ? fs.strides[q] : 1;
      if (st <= 0) break;
      for (int p = 0; p < P; p++) {
        const double al = p < c->filter_passes ? 0.5 : 0.5 * c->filter_passes + 1.0;
        std::vector<double> o(2 * R + 1, 0.0);
        for (int m = 0; m <= 2 * R; m++) {
          o[m] += al * t[m];
          if (m - st >= 0) o[m] += 0.5 * (1.0 - al) * t[m - st];
          if (m + st <= 2 * R) o[m] += 0.5 * (1.0 - al) * t[m + st];
        }
        t = o;
      }
    }
    for (int m = 0; m < 2 * FILTER_HMAX + 1; m++) taps.c[m] = m <= 2 * R ? T(t[m]) : T(0);
    taps.P = R;
    taps.s = wide ? 1 : c->filter_stride;
    // stride-1 filters of up to five taps a side take the fused x-y pass (one TMA-staged box per CTA)
    if (taps.s == 1 && taps.P >= 1 && taps.P <= 5) {
      xy_base[0] = fE; xy_base[1] = fB; xy_base[2] = J;
      xy_ok = true;
      for (int q = 0; q < 3; q++) xy_ok = xy_ok && encode_xy_map<T>(&xy_map[q], xy_base[q], g, taps.P);
      if (xy_ok) set_filter_xy_smem<T>();
    }
    tl.nt[0] = (g.n[0] + TX - 1) / TX;
    tl.nt[1] = (g.n[1] + TY - 1) / TY;
    tl.nt[2] = (g.n[2] + TZ - 1) / TZ;
    ntiles = tl.nt[0] * tl.nt[1] * tl.nt[2];
    tl.cnt = dal<int>(ntiles + 1);
    tl.start = dal<int>(ntiles + 1);
    if (!tl.cnt || !tl.start) return fail(PIC_ENOMEM, "allocation failed");
    const int smem = push3_smem<T>();
    cudaFuncSetAttribute(k3_push_tiles<T, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k3_push_tiles<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k3_push_tiles<T, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k3_push_tiles<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in 3D init");
  }

  // ---- particles --------------------------------------------------------
  int alloc_parts(long n) {
    for (int b = 0; b < 2; b++) {
      Parts3<T>& q = P2[b];
      q.x = dal<double>(n); q.y = dal<double>(n); q.z = dal<double>(n);
      q.ux = dal<T>(n); q.uy = dal<T>(n); q.uz = dal<T>(n); q.w = dal<T>(n);
      q.id = dal<uint32_t>(n); q.fl = dal<int>(n);
      if (!q.x || !q.y || !q.z || !q.ux || !q.uy || !q.uz || !q.w || !q.id || !q.fl) return PIC_ENOMEM;
    }
    if (tl.key) dfree(tl.key);
    if (tl.rank) dfree(tl.rank);
    tl.key = dal<int>(n);
    tl.rank = dal<int>(n);
    if (!tl.key || !tl.rank) return PIC_ENOMEM;
    cap = n;
    return PIC_OK;
  }

  void free_parts(Parts3<T>& q) {
    void* ps[9] = {q.x, q.y, q.z, q.ux, q.uy, q.uz, q.w, q.id, q.fl};
    for (void* p : ps) if (p) dfree(p);
    q = Parts3<T>{};
  }

  int read_count() {
    int c = 0;
    cudaMemcpyAsync(&c, &ctrl->count, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    return c;
  }

  int compact() {
    const int n_old = read_count();
    if (n_old < 0) return fail(PIC_ECUDA, "CUDA error before compaction");
    if (n_old == 0) { count_ub = 0; return PIC_OK; }
    const long nb = (n_old + 255) / 256;
    if (nb > blk_cap) {
      if (blk) dfree(blk);
      blk = dal<int>(nb);
      if (!blk) return fail(PIC_ENOMEM, "allocation failed");
      blk_cap = nb;
    }
    k3_live_per_block<<<(unsigned)nb, 256, 0, s>>>(P2[cur].fl, ctrl, blk);
    k3_scan_blocks<<<1, 1024, 0, s>>>(blk, (int)nb, ctrl);
    k3_scatter<T><<<(unsigned)nb, 256, 0, s>>>(P2[cur], P2[1 - cur], blk, n_old);
    nl += 3;
    cur = 1 - cur;
    const int n_new = read_count();
    if (n_new < 0) return fail(PIC_ECUDA, "CUDA error in compaction");
    count_ub = n_new;
    return PIC_OK;
  }

  // particles into tile order (dropping the dead ones) in the other buffer set
  void sort_tiles() {
    cudaMemsetAsync(tl.cnt, 0, sizeof(int) * (ntiles + 1), s);
    k3_tile_key<T><<<nblk(count_ub, 256), 256, 0, s>>>(g, P2[cur], ctrl, tl, (int)count_ub);
    k3_scan_tiles<<<1, 1024, 0, s>>>(tl.cnt, tl.start, ntiles, ctrl);
    k3_tile_scatter<T><<<nblk(count_ub, 256), 256, 0, s>>>(P2[cur], P2[1 - cur], tl, (int)count_ub);
    nl += 3;
    cur = 1 - cur;
    compactions++;
  }

  int grow(long need) {
    long ncap = std::max(need + need / 4, 2 * cap);
    Parts3<T> old[2] = {P2[0], P2[1]};
    const int c = read_count();
    if (c < 0) return fail(PIC_ECUDA, "CUDA error");
    P2[0] = Parts3<T>{}; P2[1] = Parts3<T>{};
    const long ocap = cap;
    if (alloc_parts(ncap) != PIC_OK) return fail(PIC_ENOMEM, "particle allocation failed");
    const Parts3<T>& o = old[cur];
    Parts3<T>& d = P2[cur];
    if (c > 0) {
      cudaMemcpyAsync(d.x, o.x, 8 * (size_t)c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.y, o.y, 8 * (size_t)c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.z, o.z, 8 * (size_t)c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.ux, o.ux, sizeof(T) * c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.uy, o.uy, sizeof(T) * c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.uz, o.uz, sizeof(T) * c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.w, o.w, sizeof(T) * c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.id, o.id, 4 * (size_t)c, cudaMemcpyDeviceToDevice, s);
      cudaMemcpyAsync(d.fl, o.fl, 4 * (size_t)c, cudaMemcpyDeviceToDevice, s);
    }
    (void)ocap;
    free_parts(old[0]);
    free_parts(old[1]);
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error while growing");
  }

  double z_hi() const { return g.hi[2] * g.d[2]; }
  double z_lo() const { return g.lo[2] * g.d[2]; }
  double time_of(long n) const { return (double)n * g.dt; }

  long long rows_inside(double t) const { return (long long)std::ceil((z_hi() + beta * kC * t) / lat.h - 0.5); }

  double row_density(long long m) const { return gamma * lab_density3(lat, gamma * ((m + 0.5) * lat.h)); }

  // create the electron rows [m0, m1) with density > 0 at time t
  int inject_rows(long long m0, long long m1, double t) {
    std::vector<long long> rows;
    for (long long m = m0; m < m1; m++)
      if (row_density(m) > 0.0) rows.push_back(m);
    const long per = (long)lat.nxl * lat.nyl;
    const long add = (long)rows.size() * per;
    if (add == 0) return PIC_OK;
    if (count_ub + add > cap) {
      if (compact() != PIC_OK) return st;
      if (count_ub + add > cap && grow(count_ub + add) != PIC_OK) return st;
    }
    for (size_t r0 = 0; r0 < rows.size(); r0 += 8) {
      Rows8 R;
      R.n = (int)std::min<size_t>(8, rows.size() - r0);
      for (int q = 0; q < R.n; q++) R.m[q] = rows[r0 + q];
      const long n = per * R.n;
      k3_inject<T><<<nblk(n, 256), 256, 0, s>>>(g, P2[cur], ctrl, lat, R, t);
      k3_add_count<<<1, 1, 0, s>>>(ctrl, (int)n);
      nl += 2;
      count_ub += n;
    }
    return PIC_OK;
  }

  int load_plasma(const pic_plasma* p) override {
    if (loaded) return fail(PIC_ESTATE, "plasma already loaded");
    const int ppc_y = p->ppc_y > 0 ? p->ppc_y : 1;
    if (p->ppc_x < 1 || p->ppc_z < 1 || p->n0 < 0) return fail(PIC_EINVAL, "bad plasma");
    lat.h = g.d[2] / p->ppc_z;
    lat.gamma = gamma; lat.beta = beta;
    lat.n0 = p->n0; lat.z_start_lab = p->z_start_lab; lat.ramp_lab = p->ramp_lab; lat.length_lab = p->length_lab;
    lat.ppc[0] = p->ppc_x; lat.ppc[1] = ppc_y; lat.ppc[2] = p->ppc_z;
    lat.nxl = (g.hi[0] - g.lo[0]) * p->ppc_x;
    lat.nyl = (g.hi[1] - g.lo[1]) * ppc_y;
    ions = p->ions != 0;
    const double t = time_of(step);
    const long long m_end = rows_inside(t);
    const long long m_beg = (long long)std::ceil((z_lo() + beta * kC * t) / lat.h - 0.5);
    const long per = (long)lat.nxl * lat.nyl;
    const long rows_box = m_end - m_beg + 1;
    const double rows_per_step = beta * kC * g.dt / lat.h + 1.0;
    long want = (long)((rows_box + rows_per_step * 64) * per * 1.1) + 1024;
    if (alloc_parts(want) != PIC_OK) return fail(PIC_ENOMEM, "particle allocation failed");
    count_ub = 0;
    if (inject_rows(m_beg, m_end, t) != PIC_OK) return st;
    row_next = m_end;
    mlo = m_beg;
    if (ions) {
      std::vector<double> tx(g.n[0] + 1, 0.0), ty(g.n[1] + 1, 0.0);
      for (int a = 0; a < lat.nxl; a++) {
        const double X = g.lo[0] + (a + 0.5) / lat.ppc[0];
        for (int i = 0; i <= g.n[0]; i++) tx[i] += shape_h(cfg.shape_order, X - i);
      }
      for (int b = 0; b < lat.nyl; b++) {
        const double Y = g.lo[1] + (b + 0.5) / lat.ppc[1];
        for (int j = 0; j <= g.n[1]; j++) ty[j] += shape_h(cfg.shape_order, Y - j);
      }
      ion_i0 = g.n[0]; ion_i1 = 0; ion_j0 = g.n[1]; ion_j1 = 0;
      for (int i = 0; i <= g.n[0]; i++)
        if (tx[i] != 0.0) { ion_i0 = std::min(ion_i0, i); ion_i1 = std::max(ion_i1, i); }
      for (int j = 0; j <= g.n[1]; j++)
        if (ty[j] != 0.0) { ion_j0 = std::min(ion_j0, j); ion_j1 = std::max(ion_j1, j); }
      if (ion_i1 < ion_i0 || ion_j1 < ion_j0) { ion_i0 = ion_i1 = ion_j0 = ion_j1 = 0; }
      Tx = dal<double>(g.n[0] + 1); Ty = dal<double>(g.n[1] + 1); Zs = dal<double>(g.n[2] + 1);
      if (!Tx || !Ty || !Zs) return fail(PIC_ENOMEM, "allocation failed");
      cudaMemcpyAsync(Tx, tx.data(), sizeof(double) * tx.size(), cudaMemcpyHostToDevice, s);
      cudaMemcpyAsync(Ty, ty.data(), sizeof(double) * ty.size(), cudaMemcpyHostToDevice, s);
      cudaStreamSynchronize(s);
    }
    // optional test beam
    if (p->beam_n > 0 && p->beam_self && !p->beam_w) return fail(PIC_EINVAL, "beam_self needs beam_w");
    if (p->beam_n > 0) {
      if (!p->beam_x || !p->beam_y || !p->beam_z || !p->beam_ux || !p->beam_uy || !p->beam_uz)
        return fail(PIC_EINVAL, "3D test beam needs x, y, z and the three momenta");
      const int n = (int)p->beam_n;
      bm.n = n;
      bm.x = dal<double>(n); bm.y = dal<double>(n); bm.z = dal<double>(n);
      bm.ux = dal<T>(n); bm.uy = dal<T>(n); bm.uz = dal<T>(n);
      bm.tc = dal<double>(n); bm.zf0 = dal<double>(n);
      bm.uxb = dal<T>(n); bm.uyb = dal<T>(n); bm.uzb = dal<T>(n); bm.fl = dal<int>(n);
      double* lab = dal<double>(6 * (size_t)n);
      if (!bm.x || !bm.fl || !lab) return fail(PIC_ENOMEM, "allocation failed");
      const double* srcs[6] = {p->beam_x, p->beam_y, p->beam_z, p->beam_ux, p->beam_uy, p->beam_uz};
      for (int q = 0; q < 6; q++)
        cudaMemcpyAsync(lab + (size_t)q * n, srcs[q], 8 * (size_t)n, cudaMemcpyHostToDevice, s);
      cudaMemsetAsync(bacc, 0, 8 * sizeof(double), s);
      k3_beam_vz<<<nblk(n, 256), 256, 0, s>>>(n, lab + 3 * (size_t)n, lab + 4 * (size_t)n, lab + 5 * (size_t)n, bacc);
      k3_beam_transform<T><<<nblk(n, 256), 256, 0, s>>>(bm, lab, lab + n, lab + 2 * (size_t)n, lab + 3 * (size_t)n,
                                                        lab + 4 * (size_t)n, lab + 5 * (size_t)n, p->beam_t_lab,
                                                        p->beam_z_plane_lab, gamma, beta, bacc);
      k3_beam_finish<T><<<nblk(n, 256), 256, 0, s>>>(bm, time_of(step), bacc);
      nl += 3;
      if (p->beam_self) {
        // self-consistent beam: weights (macro-particle counts) in the path's type
        std::vector<T> wv(n);
        for (int q = 0; q < n; q++) wv[q] = T(p->beam_w[q]);
        bm.w = dal<T>(n);
        if (!bm.w) return fail(PIC_ENOMEM, "allocation failed");
        cudaMemcpyAsync(bm.w, wv.data(), sizeof(T) * n, cudaMemcpyHostToDevice, s);
        bm.self = 1;
      }
      cudaStreamSynchronize(s);
      dfree(lab);
      has_beam = true;
    }
    loaded = true;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in 3D plasma load");
  }

  int set_laser(const pic_laser* l) override {
    if (l->beta_s != 0.0) return fail(PIC_EINVAL, "3D antenna: the plane is at rest in the computational frame");
    las = *l;
    const double om = 2.0 * kPi * kC / l->lambda0;
    E0 = l->a0 * kMe * kC * om / kQe;
    const double dop = (1.0 + beta) * gamma;
    Qpair = 200.0 * kEps0 * E0 * g.d[0] * g.d[1] / dop;
    Dn = 0.0;
    has_laser = true;
    return PIC_OK;
  }

  bool antenna_inside() const { return has_laser && las.z_antenna >= z_lo() && las.z_antenna < z_hi(); }

  // time factor of the emitted field: E_emit = G(x, y) emit_t(t'), PR-14 with beta_s = 0
  double emit_t(double tp) const {
    const double om = 2.0 * kPi * kC / las.lambda0;
    const double dop = (1.0 + beta) * gamma;
    const double sl = tp / dop;
    const double sig = las.tau_fwhm / (2.0 * std::sqrt(std::log(2.0)));
    return E0 * std::exp(-(sl - las.t_peak) * (sl - las.t_peak) / (2.0 * sig * sig)) *
           std::sin(om * (sl - las.t_peak) + las.phase) / dop;
  }

  Ant3 ant_params(double D0, double D1) const {
    Ant3 a;
    a.x_center = las.x_center; a.y_center = las.y_center; a.w0 = las.w0; a.za = las.z_antenna;
    a.D0 = D0; a.D1 = D1; a.Q = Qpair; a.order = cfg.shape_order;
    return a;
  }

  // ---- one step (order of PR-1) ------------------------------------------
  void btd_part(int which, int post) {
    if (rz.empty()) return;
    const long plane = (long)(g.n[0] + 1) * (g.n[1] + 1);
    for (size_t r = 0; r < rz.size(); r++) {
      const double tp = gamma * (rt[r] - beta * rz[r] / kC);
      const double zp = gamma * (rz[r] - beta * kC * rt[r]);
      double ta, tb;
      if (which == 0) { ta = time_of(step); tb = time_of(step + 1); }
      else { ta = time_of(step) - 0.5 * g.dt; tb = ta + g.dt; }
      if (!(tp >= ta && tp < tb)) continue;
      const double f = (tp - ta) / g.dt;
      const double wgt = post ? f : 1.0 - f;
      k3_btd<T><<<nblk(plane, 256), 256, 0, s>>>(g, E, B, rout + r * 6 * plane, which, wgt, zp, gamma, beta);
      nl++;
      if (post) rdone[2 * r + which] = 1;
    }
  }

  dim3 grid3() const { return dim3(nblk(g.n[2] + 1, 128 * KPT), g.n[1] + 1, g.n[0] + 1); }

  void filter3(T* F, int comp) {
    // F inside one of the mapped blocks: x and y in one TMA-staged pass F -> tmp, then z: tmp -> F
    for (int q = 0; xy_ok && q < 3; q++) {
      const long d = F - xy_base[q];
      if (d < 0 || d >= 3 * g.cs || d % g.cs != 0) continue;
      const int slot = (int)(d / g.cs);
      switch (taps.P) {
        case 1: launch_filter_xy<T, 1>(g, xy_map[q], slot, tmp, comp, taps, ctrl, s); break;
        case 2: launch_filter_xy<T, 2>(g, xy_map[q], slot, tmp, comp, taps, ctrl, s); break;
        case 3: launch_filter_xy<T, 3>(g, xy_map[q], slot, tmp, comp, taps, ctrl, s); break;
        case 4: launch_filter_xy<T, 4>(g, xy_map[q], slot, tmp, comp, taps, ctrl, s); break;
        default: launch_filter_xy<T, 5>(g, xy_map[q], slot, tmp, comp, taps, ctrl, s); break;
      }
      launch_filter_axis<T>(g, grid3(), tmp, F, comp, 2, taps, s);
      nl += 2;
      return;
    }
    // x: F -> tmp, y: tmp -> tmp2, z: tmp2 -> F
    launch_filter_axis<T>(g, grid3(), F, tmp, comp, 0, taps, s);
    launch_filter_axis<T>(g, grid3(), tmp, tmp2, comp, 1, taps, s);
    launch_filter_axis<T>(g, grid3(), tmp2, F, comp, 2, taps, s);
    nl += 3;
  }

  // CUDA events around the launches of the timed kernel class (host waits for the end event)
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
    const long nn = nodes();
    const long n3 = 3 * g.cs;
    const double th = cfg.theta;
    btd_part(0, 0);
    btd_part(1, 0);
    // 1. Faraday + Friedman + PML-B (B^{n-1/2} -> B^{n+1/2}), gather copies
    tbeg(1);
    k3_faraday_tile<T><<<dim3(nblk(g.n[2] + 1, FZ), nblk(g.n[1] + 1, FY), nblk(g.n[0] + 1, FX)), dim3(FZ, FY), 0, s>>>(
        g, pm, E, Ep, Eb, B, Bs, fB, T(1.0 + th / 4.0), T(0.5), T(0.5 - th / 4.0), T(cfg.ck_alpha), T(cfg.ck_beta),
        T(cfg.ck_gamma), T(g.dt));
    k3_friedman<T><<<nblk(n3, 256), 256, 0, s>>>(n3, E, Ep, Eb, fE, T(1.0 - th / 2.0), T(th / 2.0));
    nl += 2;
    if (cfg.filter_gather && P > 0)
      for (int c = 0; c < 3; c++) { filter3(fE + c * g.cs, c); filter3(fB + c * g.cs, 3 + c); }
    tend(1);
    // 2. particles
    cudaMemsetAsync(J, 0, sizeof(T) * 3 * g.cs, s);
    Fld3<T> f;
    for (int c = 0; c < 3; c++) { f.fE[c] = fE + c * g.cs; f.fB[c] = fB + c * g.cs; f.J[c] = J + c * g.cs; }
    if (nodal) {
      // 'momentum conserving' gather: the copies interpolated to the nodes
      k3_nodal<T><<<grid3(), 128, 0, s>>>(g, fE, fB, nF);
      nl++;
      for (int c = 0; c < 3; c++) { f.fE[c] = nF + c * g.cs; f.fB[c] = nF + (3 + c) * g.cs; }
    }
    const T kq = T(-kQe * g.dt / (2.0 * kMe));
    if (loaded && count_ub > 0) {
      sort_tiles();
      const int smem = push3_smem<T>();
      tbeg(0);
      if (cfg.shape_order == 3 && !nodal)
        k3_push_tiles<T, 3, false><<<ntiles, 256, smem, s>>>(g, f, P2[cur], tl, ctrl, kq, cq_e);
      else if (cfg.shape_order == 3)
        k3_push_tiles<T, 3, true><<<ntiles, 256, smem, s>>>(g, f, P2[cur], tl, ctrl, kq, cq_e);
      else if (!nodal)
        k3_push_tiles<T, 1, false><<<ntiles, 256, smem, s>>>(g, f, P2[cur], tl, ctrl, kq, cq_e);
      else
        k3_push_tiles<T, 1, true><<<ntiles, 256, smem, s>>>(g, f, P2[cur], tl, ctrl, kq, cq_e);
      nl++;
      tend(0);
    }
    const double tn = time_of(step), tn1 = time_of(step + 1);
    if (loaded && ions && row_next > mlo) {
      k3_ion_z<<<nblk(g.n[2] + 1, 4), 128, 0, s>>>(g, lat, cfg.shape_order, mlo, row_next, tn, tn1, Zs);
      k3_ion_jz<T><<<dim3(nblk(g.n[2] + 1, 128 * KPT), ion_j1 - ion_j0 + 1, ion_i1 - ion_i0 + 1), 128, 0, s>>>(
          g, Tx, Ty, Zs, -kQe / (g.d[0] * g.d[1] * g.dt), ion_i0, ion_j0, J + 2 * g.cs);
      nl += 2;
    }
    if (has_beam) {
      if (cfg.shape_order == 3)
        k3_beam_push<T, 3><<<nblk(bm.n, 128), 128, 0, s>>>(g, f, bm, tn, tn1, bacc, kq, nodal ? 1 : 0);
      else
        k3_beam_push<T, 1><<<nblk(bm.n, 128), 128, 0, s>>>(g, f, bm, tn, tn1, bacc, kq, nodal ? 1 : 0);
      nl++;
    }
    // 3. antenna: the moving partners' displacement G(x, y) D_n -> G D_{n+1}
    if (antenna_inside()) {
      const double th_ = tn + 0.5 * g.dt;
      const double dD = -2.0 * kEps0 * kC * emit_t(th_) * g.d[0] * g.d[1] / Qpair * g.dt;
      const Ant3 a = ant_params(Dn, Dn + dD);
      const int npair = (g.hi[0] - g.lo[0] + 1) * (g.hi[1] - g.lo[1] + 1);
      k3_antenna<T><<<nblk(npair, 128), 128, 0, s>>>(g, J + g.cs, a);
      nl++;
      Dn += dD;
    }
    // 4. current filter, Ampere + PML-E
    tbeg(1);
    if (cfg.filter_J && P > 0)
      for (int c = 0; c < 3; c++) filter3(J + c * g.cs, c);
    k3_ampere<T><<<grid3(), 128, 0, s>>>(g, pm, E, Es, B, J, T(g.dt * kC * kC), T(g.dt / kEps0));
    nl++;
    tend(1);
    btd_part(0, 1);
    btd_part(1, 1);
    // 5. ion rows that left the particle domain, inflow through z_hi
    if (loaded) {
      while (mlo < row_next && (mlo + 0.5) * lat.h - beta * kC * tn1 < z_lo()) mlo++;
      const long long m_end = rows_inside(tn1);
      if (m_end > row_next) {
        if (inject_rows(row_next, m_end, tn1) != PIC_OK) return st;
        row_next = m_end;
      }
    }
    step++;
    return PIC_OK;
  }

  int run(int n) override {
    if (st != PIC_OK) return st;
    for (int q = 0; q < n; q++)
      if (one_step() != PIC_OK) return st;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in 3D step");
  }

  int sync() override {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(PIC_ECUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
    int dst = 0;
    cudaMemcpy(&dst, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (dst & ST_OUTSIDE) return fail(PIC_EOVERFLOW, "a particle left its tile's window (not pushed)");
    if (dst & ST_TIMEOUT) return fail(PIC_ETIMEOUT, "a bounded wait for a staged filter box gave up");
    return st;
  }

  // ---- lab-frame samples -------------------------------------------------
  int btd_set(const pic_btd_req* r) override {
    if (r->n_rows <= 0 || !r->z_lab || !r->t_lab) return fail(PIC_EINVAL, "empty lab-sample request");
    rz.assign(r->z_lab, r->z_lab + r->n_rows);
    rt.assign(r->t_lab, r->t_lab + r->n_rows);
    rdone.assign(2 * r->n_rows, 0);
    if (rout) dfree(rout);
    rout = dal<T>((size_t)r->n_rows * 6 * (g.n[0] + 1) * (g.n[1] + 1));
    return rout ? PIC_OK : fail(PIC_ENOMEM, "allocation failed");
  }

  int btd_get(pic_btd_out* o) override {
    if (!rout) return fail(PIC_ESTATE, "no lab-sample request");
    const size_t n = rz.size() * 6 * (size_t)(g.n[0] + 1) * (g.n[1] + 1);
    if (o->data)
      cudaMemcpyAsync(o->data, rout, n * sizeof(T), o->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    long long filled = 0;
    for (size_t r = 0; r < rz.size(); r++) filled += rdone[2 * r] && rdone[2 * r + 1];
    if (o->done)
      cudaMemcpyAsync(o->done, rdone.data(), sizeof(int) * rdone.size(),
                      o->on_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, s);
    o->n_rows_filled = filled;
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in btd_get");
  }

  // ---- accessors -----------------------------------------------------------
  const T* comp_ptr(int comp) const {
    if (comp < 3) return E + comp * g.cs;
    if (comp < 6) return B + (comp - 3) * g.cs;
    return J + (comp - 6) * g.cs;
  }

  int get_field(int comp, double* dst, int on_device) override {
    if (comp < 0 || comp > PIC_RHO) return fail(PIC_EINVAL, "bad component");
    const long nn = nodes();
    if (!out_d) { out_d = dal<double>(nn); if (!out_d) return fail(PIC_ENOMEM, "allocation failed"); }
    if (comp == PIC_RHO) {
      if (!rho) { rho = dal<double>(g.cs); if (!rho) return fail(PIC_ENOMEM, "allocation failed"); }
      cudaMemsetAsync(rho, 0, sizeof(double) * g.cs, s);
      if (loaded && count_ub > 0) {
        k3_particle_rho<T><<<nblk(count_ub, 128), 128, 0, s>>>(g, P2[cur], ctrl, cfg.shape_order, -kQe, rho);
        nl++;
      }
      if (loaded && ions && row_next > mlo) {
        k3_ion_rho<<<nblk(nn, 128), 128, 0, s>>>(g, lat, cfg.shape_order, mlo, row_next, time_of(step), Tx, Ty, rho);
        nl++;
      }
      if (antenna_inside() && Dn != 0.0) {
        const int npair = (g.hi[0] - g.lo[0] + 1) * (g.hi[1] - g.lo[1] + 1);
        k3_antenna_rho<<<nblk(npair, 128), 128, 0, s>>>(g, ant_params(Dn, Dn), rho);
        nl++;
      }
      k3_out_rho<<<nblk(nn, 256), 256, 0, s>>>(g, rho, out_d);
    } else {
      k3_out_field<T><<<nblk(nn, 256), 256, 0, s>>>(g, comp_ptr(comp), out_d);
    }
    nl++;
    cudaMemcpyAsync(dst, out_d, sizeof(double) * nn, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s);
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in get_field");
  }

  // the frozen beam's self-field (Sec. 3.1.1, PR-27) solved on the device: E from the positions now, B_x, B_y
  // from the positions half a step earlier (B^{n-1/2})
  int beam_self_field() override {
    if (!has_beam || !bm.self) return fail(PIC_ESTATE, "pic_beam_self_field: no self-consistent test beam");
    if (g.n[0] < 2 || g.n[1] < 2 || g.n[2] < 2) return fail(PIC_EINVAL, "pic_beam_self_field: grid too small");
    const long nn = nodes();
    const long L = g.n[2] + 1, PL = (long)(g.n[1] + 1) * L;
    double* a = dal<double>(nn);
    double* b = dal<double>(nn);
    double* tab[3];
    for (int q = 0; q < 3; q++) tab[q] = dal<double>(2 * (size_t)g.n[q]);
    if (!a || !b || !tab[0] || !tab[1] || !tab[2]) return fail(PIC_ENOMEM, "pic_beam_self_field: allocation failed");
    for (int q = 0; q < 3; q++) {
      std::vector<double> t(2 * (size_t)g.n[q]);
      for (int m = 0; m < 2 * g.n[q]; m++) t[m] = std::sin(kPi * m / g.n[q]);
      cudaMemcpyAsync(tab[q], t.data(), t.size() * 8, cudaMemcpyHostToDevice, s);
    }
    double v = 0.0;
    cudaMemcpyAsync(&v, bacc + 2, sizeof(double), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    const double gv2 = 1.0 / (1.0 - (v / kC) * (v / kC));
    auto dst = [&](const double* in, double* out, int axis) {
      const int nx1 = g.n[0] + 1, ny1 = g.n[1] + 1, nz1 = g.n[2] + 1;
      long cnt;
      if (axis == 2) {
        cnt = (long)(g.n[2] - 1) * (nx1 - 2) * (ny1 - 2);
        k3_dst<<<nblk(cnt, 256), 256, 0, s>>>(in, out, tab[2], g.n[2], nx1, ny1, PL, L, 1);
      } else if (axis == 1) {
        cnt = (long)(g.n[1] - 1) * (nx1 - 2) * (nz1 - 2);
        k3_dst<<<nblk(cnt, 256), 256, 0, s>>>(in, out, tab[1], g.n[1], nx1, nz1, PL, 1, L);
      } else {
        cnt = (long)(g.n[0] - 1) * (ny1 - 2) * (nz1 - 2);
        k3_dst<<<nblk(cnt, 256), 256, 0, s>>>(in, out, tab[0], g.n[0], ny1, nz1, L, 1, PL);
      }
    };
    const long ni = (long)(g.n[0] - 1) * (g.n[1] - 1) * (g.n[2] - 1);
    for (int mode = 0; mode < 2; mode++) {
      cudaMemsetAsync(a, 0, sizeof(double) * nn, s);
      cudaMemsetAsync(b, 0, sizeof(double) * nn, s);
      const int ord = cfg.shape_order;
      k3_beam_rho<T><<<nblk(bm.n, 128), 128, 0, s>>>(g, bm, ord, mode == 0 ? 0.0 : -0.5 * g.dt, bacc, a);
      dst(a, b, 2); dst(b, a, 1); dst(a, b, 0);
      k3_poisson_divide<<<nblk(ni, 256), 256, 0, s>>>(b, g, gv2);
      dst(b, a, 2); dst(a, b, 1); dst(b, a, 0);
      k3_zero_faces<<<nblk(nn, 256), 256, 0, s>>>(a, g);
      k3_self_field_add<T><<<nblk(nn, 256), 256, 0, s>>>(g, E, B, a, gv2, bacc, mode);
      nl += 10;
    }
    cudaStreamSynchronize(s);
    for (int q = 2; q >= 0; q--) dfree(tab[q]);
    dfree(b);
    dfree(a);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in pic_beam_self_field");
  }

  int set_field(int comp, const double* src) override {
    if (comp < 0 || comp > 8) return fail(PIC_EINVAL, "bad component");
    const long nn = nodes();
    if (!out_d) { out_d = dal<double>(nn); if (!out_d) return fail(PIC_ENOMEM, "allocation failed"); }
    cudaMemcpyAsync(out_d, src, sizeof(double) * nn, cudaMemcpyHostToDevice, s);
    k3_in_field<T><<<nblk(nn, 256), 256, 0, s>>>(g, out_d, const_cast<T*>(comp_ptr(comp)));
    nl++;
    return cudaStreamSynchronize(s) == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in set_field");
  }

  int get_particles(int species, double* x, double* y, double* z, double* ux, double* uy, double* uz, double* w,
                    uint32_t* id, int32_t* flags, int64_t* count) override {
    if (species != PIC_ELECTRONS && species != PIC_BEAM) return fail(PIC_EINVAL, "bad species");
    std::vector<int> fl;
    long n = 0;
    const bool el = species == PIC_ELECTRONS;
    if (el) {
      if (!loaded) { *count = 0; return PIC_OK; }
      n = read_count();
      if (n < 0) return fail(PIC_ECUDA, "CUDA error");
    } else {
      n = has_beam ? bm.n : 0;
    }
    fl.resize(n);
    if (n) cudaMemcpy(fl.data(), el ? P2[cur].fl : bm.fl, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    long live = 0;
    for (long q = 0; q < n; q++) live += (fl[q] & 1) != 0;
    if (!x && !y && !z && !ux && !uy && !uz && !w && !id && !flags) { *count = live; return PIC_OK; }
    if (*count < live) return fail(PIC_EINVAL, "output capacity too small");
    std::vector<double> vd(n);
    std::vector<T> vt(n);
    std::vector<uint32_t> vi(n);
    auto pickd = [&](const double* src, double* dst) {
      if (!dst || !n) return;
      cudaMemcpy(vd.data(), src, 8 * (size_t)n, cudaMemcpyDeviceToHost);
      long o = 0;
      for (long q = 0; q < n; q++) if (fl[q] & 1) dst[o++] = vd[q];
    };
    auto pickt = [&](const T* src, double* dst) {
      if (!dst || !n) return;
      cudaMemcpy(vt.data(), src, sizeof(T) * (size_t)n, cudaMemcpyDeviceToHost);
      long o = 0;
      for (long q = 0; q < n; q++) if (fl[q] & 1) dst[o++] = (double)vt[q];
    };
    if (el) {
      const Parts3<T>& p = P2[cur];
      pickd(p.x, x); pickd(p.y, y); pickd(p.z, z); pickt(p.ux, ux); pickt(p.uy, uy); pickt(p.uz, uz); pickt(p.w, w);
      if (id && n) {
        cudaMemcpy(vi.data(), p.id, 4 * (size_t)n, cudaMemcpyDeviceToHost);
        long o = 0;
        for (long q = 0; q < n; q++) if (fl[q] & 1) id[o++] = vi[q];
      }
    } else {
      pickd(bm.x, x); pickd(bm.y, y); pickd(bm.z, z); pickt(bm.ux, ux); pickt(bm.uy, uy); pickt(bm.uz, uz);
      if (w) { long o = 0; for (long q = 0; q < n; q++) if (fl[q] & 1) w[o++] = 1.0; }
      if (id) { long o = 0; for (long q = 0; q < n; q++) if (fl[q] & 1) id[o++] = (uint32_t)q; }
    }
    if (flags) { long o = 0; for (long q = 0; q < n; q++) if (fl[q] & 1) flags[o++] = fl[q]; }
    *count = live;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : fail(PIC_ECUDA, "CUDA error in get_particles");
  }

  int stats(pic_stats* o) override {
    double trap = o->trap_gamma_lab > 0.0 ? o->trap_gamma_lab : 0.0;
    if (trap == 0.0 && has_laser && loaded && lat.n0 > 0.0) {
      const double wp = std::sqrt(lat.n0 * kQe * kQe / (kEps0 * kMe));
      trap = 2.0 * (2.0 * kPi * kC / las.lambda0) / wp;
    }
    cudaMemsetAsync(sred, 0, 8 * sizeof(double), s);
    k3_stats<T><<<152 * 8, 256, 0, s>>>(g, E, B, P2[cur], ctrl, bm, gamma, beta, trap, sred);
    nl++;
    double h[8];
    cudaMemcpyAsync(h, sred, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(PIC_ECUDA, "CUDA error in stats");
    o->step = step; o->t = time_of(step);
    o->dt = g.dt; o->dx = g.d[0]; o->dz = g.d[2]; o->gamma = gamma; o->beta = beta;
    o->n_electrons = loaded ? (int64_t)h[0] : 0;
    o->n_beam_active = (int64_t)h[1];
    o->beam_gamma_lab = h[1] > 0 ? h[2] / h[1] : 0.0;
    const double var = h[1] > 0 ? h[3] / h[1] - o->beam_gamma_lab * o->beam_gamma_lab : 0.0;
    o->beam_spread = o->beam_gamma_lab > 0 ? std::sqrt(var > 0 ? var : 0) / o->beam_gamma_lab : 0.0;
    o->field_energy = h[4];
    o->gx_lo = g.lo[0]; o->gx_hi = g.hi[0]; o->gz_lo = g.lo[2]; o->gz_hi = g.hi[2];
    o->sorts = compactions; o->overflow_chunks = 0;
    o->z0 = 0.0;
    o->trap_gamma_lab = trap;
    o->trapped_charge = kQe * h[5];
    return PIC_OK;
  }

  int64_t launches() const override { return nl; }

  int kernel_timing(int enable, int which, double* ms_total, int64_t* n) override {
    if (which != 0 && which != 1) return PIC_EINVAL;
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
};

}  // namespace

Sim3Api* make_sim3(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* user, cudaStream_t s,
                   int* status, std::string* err) {
  if (cfg->ny < 8 || !(cfg->dy > 0)) {
    *status = PIC_EINVAL;
    if (err) *err = "3D needs ny >= 8 and dy > 0";
    return nullptr;
  }
  if (cfg->moving_window) {
    *status = PIC_EINVAL;
    if (err) *err = "3D runs have no moving window";
    return nullptr;
  }
  Sim3Api* r = nullptr;
  int rc;
  if (cfg->precision == PIC_FP64) {
    auto* p = new Sim3<double>();
    p->s = s; p->alloc = alloc; p->freef = free_fn; p->user = user;
    rc = p->init(cfg);
    r = p;
  } else {
    auto* p = new Sim3<float>();
    p->s = s; p->alloc = alloc; p->freef = free_fn; p->user = user;
    rc = p->init(cfg);
    r = p;
  }
  if (rc != PIC_OK) {
    if (err) *err = r->error();
    delete r;
    *status = rc;
    return nullptr;
  }
  *status = PIC_OK;
  return r;
}

}  // namespace picgb
