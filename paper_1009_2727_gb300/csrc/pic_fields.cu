// Field kernels of the boosted-frame PIC step:
//  - Faraday with the tunable (Cole-Karkkainen) operator, Friedman damping and
//    the split-field PML for B (Eq. Faraday, Eq. Faraday_Friedman, App. II);
//  - the multi-pass bilinear filter with compensation (Sec. 4.1), applied to
//    the fields used by the gather, tile by tile in shared memory;
//  - Ampere with the Yee operator and the split-field PML for E, fused with the
//    filter of the deposited current and the rigid ion-column current.
#include "pic_common.cuh"

namespace picgb {

namespace {

template <class T>
struct FarK {
  T a2, b2;          // 2D reduced coefficients: alpha + 2 beta, beta + 2 gamma
  T c1, c2, c3;      // E_eff = c1 E^n + c2 E^{n-1} + c3 E-bar
  T h1, h2;          // E-bar' = h1 E^n + h2 E-bar
};

template <class T, bool FRIED>
__device__ __forceinline__ T eeff(const FieldPtrs<T>& f, const FarK<T>& q, const GridP& g, int c, int i, int k) {
  if (i < 0 || i > g.nx || k < 0 || k > g.nz) return T(0);
  const long p = (long)i * g.ld + k;
  T e = f.E[c][p];
  if (FRIED) e = q.c1 * e + q.c2 * f.Eo[c][p] + q.c3 * f.Eb[c][p];
  return e;
}

// Delta*_z at (i, k+1/2) of a field sampled at k, smoothed over x-neighbours (PR-2, PR-3)
template <class T, bool FRIED, bool CK>
__device__ __forceinline__ T dstar_z(const FieldPtrs<T>& f, const FarK<T>& q, const GridP& g, int c, int i, int k) {
  T d0 = eeff<T, FRIED>(f, q, g, c, i, k + 1) - eeff<T, FRIED>(f, q, g, c, i, k);
  if (!CK) return d0 / T(g.dz);
  T dp = eeff<T, FRIED>(f, q, g, c, i + 1, k + 1) - eeff<T, FRIED>(f, q, g, c, i + 1, k);
  T dm = eeff<T, FRIED>(f, q, g, c, i - 1, k + 1) - eeff<T, FRIED>(f, q, g, c, i - 1, k);
  return (q.a2 * d0 + q.b2 * (dp + dm)) / T(g.dz);
}

template <class T, bool FRIED, bool CK>
__device__ __forceinline__ T dstar_x(const FieldPtrs<T>& f, const FarK<T>& q, const GridP& g, int c, int i, int k) {
  T d0 = eeff<T, FRIED>(f, q, g, c, i + 1, k) - eeff<T, FRIED>(f, q, g, c, i, k);
  if (!CK) return d0 / T(g.dx);
  T dp = eeff<T, FRIED>(f, q, g, c, i + 1, k + 1) - eeff<T, FRIED>(f, q, g, c, i, k + 1);
  T dm = eeff<T, FRIED>(f, q, g, c, i + 1, k - 1) - eeff<T, FRIED>(f, q, g, c, i, k - 1);
  return (q.a2 * d0 + q.b2 * (dp + dm)) / T(g.dx);
}

template <class T, bool FRIED, bool CK>
__global__ void __launch_bounds__(256) k_faraday(GridP g, FieldPtrs<T> f, PmlTabs pt, FarK<T> q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y * blockDim.y + threadIdx.y;
  if (i > g.nx || k > g.nz) return;
  const long p = (long)i * g.ld + k;
  const T dt = T(g.dt);
  // Bx at (i, k+1/2): dBx/dt = Delta*_z Ey
  if (k <= g.nz - 1) {
    T d = dstar_z<T, FRIED, CK>(f, q, g, EY, i, k);
    T bo = f.B[0][p], bn;
    double sz = pt.sz_h[k];
    if (sz > 0.0) bn = T(pt.xz_h[k] * (double)bo + pt.cz_h[k] * (double)d);
    else bn = bo + dt * d;
    f.B[0][p] = bn;
    f.Bavg[0][p] = T(0.5) * (bo + bn);
  }
  // Bz at (i+1/2, k): dBz/dt = -Delta*_x Ey
  if (i <= g.nx - 1) {
    T d = dstar_x<T, FRIED, CK>(f, q, g, EY, i, k);
    T bo = f.B[2][p], bn;
    double sx = pt.sx_h[i];
    if (sx > 0.0) bn = T(pt.xx_h[i] * (double)bo - pt.cx_h[i] * (double)d);
    else bn = bo - dt * d;
    f.B[2][p] = bn;
    f.Bavg[2][p] = T(0.5) * (bo + bn);
  }
  // By at (i+1/2, k+1/2): dBy/dt = -Delta*_z Ex + Delta*_x Ez; split in the PML
  if (i <= g.nx - 1 && k <= g.nz - 1) {
    T a = dstar_z<T, FRIED, CK>(f, q, g, EX, i, k);
    T b = dstar_x<T, FRIED, CK>(f, q, g, EZ, i, k);
    T bo = f.B[1][p], bn;
    double sx = pt.sx_h[i], sz = pt.sz_h[k];
    if (sx > 0.0 || sz > 0.0) {
      double yz = pt.xz_h[k] * (double)f.Byz[p] - pt.cz_h[k] * (double)a;
      double yx = pt.xx_h[i] * (double)f.Byx[p] + pt.cx_h[i] * (double)b;
      f.Byz[p] = T(yz);
      f.Byx[p] = T(yx);
      bn = T(yx) + T(yz);
    } else {
      bn = bo - dt * (a - b);
    }
    f.B[1][p] = bn;
    f.Bavg[1][p] = T(0.5) * (bo + bn);
  }
  if (FRIED) {
#pragma unroll
    for (int c = 0; c < 3; c++) f.Ebn[c][p] = q.h1 * f.E[c][p] + q.h2 * f.Eb[c][p];
  }
}

// ---------------------------------------------------------------------------
// Shared-memory tile filter. The n bilinear passes and the compensation pass of
// Sec. 4.1 along one axis compose into one (2P+1)-tap convolution with taps at
// multiples of the stride (P = n + compensation); the separable 2D filter is that
// convolution along x, then along z. Away from the walls this is the pass-by-pass
// filter up to rounding; within P*stride cells of a wall the pass-by-pass filter
// would also re-zero values outside each component's valid range, but no particle
// reads there and the deposited current is zero there (PR-6, PR-10), which the
// particle guard enforces.
constexpr int FT_X = 16;
constexpr int FT_Z = 64;
constexpr int FT_TY = 4;

template <class T>
__device__ __forceinline__ void load_tile(T* A, const T* src, const GridP& g, int gi0, int gk0, int WX, int WZ,
                                          const double* ion_x, const double* ion_c, double ion_coef) {
  for (int li = threadIdx.y; li < WX; li += FT_TY) {
    const int gi = gi0 + li;
    const bool rowok = gi >= 0 && gi <= g.nx;
    const double ix = (rowok && ion_x) ? ion_coef * ion_x[gi] : 0.0;
    for (int lk = threadIdx.x; lk < WZ; lk += FT_Z) {
      const int gk = gk0 + lk;
      T v = T(0);
      if (rowok && gk >= 0 && gk <= g.nz) {
        v = src[(long)gi * g.ld + gk];
        if (ion_x) v += T(ix * ion_c[gk]);
      }
      A[li * WZ + lk] = v;
    }
  }
}

// x-pass: B1[ti][lk] = sum_j c_j A[ti + H + (j - P) s][lk] for the tile's rows
template <class T>
__device__ __forceinline__ void xpass(const T* A, T* B1, const FilterTaps<T>& ft, int WZ) {
  for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
    for (int lk = threadIdx.x; lk < WZ; lk += FT_Z) {
      const T* col = A + (ti + ft.H - ft.P * ft.s) * WZ + lk;
      T acc = T(0);
      for (int j = 0; j <= 2 * ft.P; j++) acc += ft.c[j] * col[j * ft.s * WZ];
      B1[ti * WZ + lk] = acc;
    }
  }
}

// z-pass value at (ti, tk)
template <class T>
__device__ __forceinline__ T zpass(const T* B1, const FilterTaps<T>& ft, int WZ, int ti, int tk) {
  const T* row = B1 + ti * WZ + tk + ft.H - ft.P * ft.s;
  T acc = T(0);
  for (int j = 0; j <= 2 * ft.P; j++) acc += ft.c[j] * row[j * ft.s];
  return acc;
}

// gather copies: fE = F(E^n), fB = F(Bavg)
template <class T>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_filter_fields(GridP g, FieldPtrs<T> f, FilterTaps<T> ft) {
  extern __shared__ unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);
  const int H = ft.H;
  const int WX = FT_X + 2 * H, WZ = FT_Z + 2 * H;
  T* B1 = A + WX * WZ;
  const int i0 = blockIdx.y * FT_X, k0 = blockIdx.x * FT_Z;
  for (int c = 0; c < 6; c++) {
    const T* src = c < 3 ? f.E[c] : f.Bavg[c - 3];
    T* dst = c < 3 ? f.fE[c] : f.fB[c - 3];
    load_tile<T>(A, src, g, i0 - H, k0 - H, WX, WZ, nullptr, nullptr, 0.0);
    __syncthreads();
    xpass<T>(A, B1, ft, WZ);
    __syncthreads();
    const int gk = k0 + threadIdx.x;
    for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
      const int gi = i0 + ti;
      const T v = zpass<T>(B1, ft, WZ, ti, threadIdx.x);
      if (gi <= g.nx && gk <= g.nz) dst[(long)gi * g.ld + gk] = v;
    }
    __syncthreads();
  }
}

// Ampere + PML-E, with the current (plus the ion column current) filtered in the tile first
template <class T, bool FILT>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_ampere(GridP g, FieldPtrs<T> f, PmlTabs pt, FilterTaps<T> ft,
                                                        const double* ion_x, const double* ion_c, double ion_coef) {
  extern __shared__ unsigned char smraw[];
  T* A = reinterpret_cast<T*>(smraw);
  const int H = FILT ? ft.H : 0;
  const int WX = FT_X + 2 * H, WZ = FT_Z + 2 * H;
  T* B1 = A + WX * WZ;
  const int i0 = blockIdx.y * FT_X, k0 = blockIdx.x * FT_Z;
  const T dt = T(g.dt);
  const T c2 = T(kC * kC);
  const T ie0 = T(1.0 / kEps0);
  const double c2d = kC * kC;
  const int k = k0 + threadIdx.x;
  for (int c = 0; c < 3; c++) {
    int vi0, vi1, vk0, vk1;
    valid_range(c, g.nx, g.nz, vi0, vi1, vk0, vk1);
    const bool ion = (c == 2) && ion_x != nullptr;
    load_tile<T>(A, f.J[c], g, i0 - H, k0 - H, WX, WZ, ion ? ion_x : nullptr, ion_c, ion_coef);
    __syncthreads();
    if (FILT) {
      xpass<T>(A, B1, ft, WZ);
      __syncthreads();
    }
    for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
      const int i = i0 + ti;
      if (i > g.nx || k > g.nz) continue;
      const long p = (long)i * g.ld + k;
      f.Jn[c][p] = T(0);
      const bool v = i >= vi0 && i <= vi1 && k >= vk0 && k <= vk1;
      if (!v) { f.Eo[c][p] = T(0); continue; }
      const T jv = FILT ? zpass<T>(B1, ft, WZ, ti, threadIdx.x) : A[ti * WZ + threadIdx.x];
      const T eo = f.E[c][p];
      T en;
      if (c == 0) {
        T d = (f.B[1][p] - f.B[1][p - 1]) / T(g.dz);
        double sz = pt.sz_i[k];
        if (sz > 0.0) en = T(pt.xz_i[k] * (double)eo - c2d * pt.cz_i[k] * (double)d);
        else en = eo - dt * (c2 * d + jv * ie0);
      } else if (c == 2) {
        T d = (f.B[1][p] - f.B[1][p - g.ld]) / T(g.dx);
        double sx = pt.sx_i[i];
        if (sx > 0.0) en = T(pt.xx_i[i] * (double)eo + c2d * pt.cx_i[i] * (double)d);
        else en = eo + dt * (c2 * d - jv * ie0);
      } else {
        T dbx = (f.B[0][p] - f.B[0][p - 1]) / T(g.dz);
        T dbz = (f.B[2][p] - f.B[2][p - g.ld]) / T(g.dx);
        double sx = pt.sx_i[i], sz = pt.sz_i[k];
        if (sx > 0.0 || sz > 0.0) {
          double yz = pt.xz_i[k] * (double)f.Eyz[p] + c2d * pt.cz_i[k] * (double)dbx;
          double yx = pt.xx_i[i] * (double)f.Eyx[p] - c2d * pt.cx_i[i] * (double)dbz;
          f.Eyz[p] = T(yz);
          f.Eyx[p] = T(yx);
          en = T(yx) + T(yz);
        } else {
          en = eo + dt * (c2 * (dbx - dbz) - jv * ie0);
        }
      }
      f.Eo[c][p] = en;
    }
    __syncthreads();
  }
}

}  // namespace

template <class T>
void launch_faraday(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, double a2, double b2, double theta,
                    bool friedman, cudaStream_t s) {
  FarK<T> q;
  q.a2 = T(a2); q.b2 = T(b2);
  q.c1 = T(1.0 + theta / 4.0); q.c2 = T(-0.5); q.c3 = T(0.5 - theta / 4.0);
  q.h1 = T(1.0 - theta / 2.0); q.h2 = T(theta / 2.0);
  dim3 blk(32, 8), grd((g.nz + 1 + 31) / 32, (g.nx + 1 + 7) / 8);
  const bool ck = b2 != 0.0;
  if (friedman) {
    if (ck) k_faraday<T, true, true><<<grd, blk, 0, s>>>(g, f, pt, q);
    else k_faraday<T, true, false><<<grd, blk, 0, s>>>(g, f, pt, q);
  } else {
    if (ck) k_faraday<T, false, true><<<grd, blk, 0, s>>>(g, f, pt, q);
    else k_faraday<T, false, false><<<grd, blk, 0, s>>>(g, f, pt, q);
  }
}

static size_t tile_smem(int H, size_t elem) {
  return ((size_t)(FT_X + 2 * H) * (FT_Z + 2 * H) + (size_t)FT_X * (FT_Z + 2 * H)) * elem;
}

template <class T>
static FilterTaps<T> make_taps(const FilterSpec& fs) {
  // compose n bilinear passes (alpha = 1/2) and the compensation pass (alpha_c = n/2 + 1)
  double k[2 * 16 + 1] = {0.0};
  int len = 1;
  k[0] = 1.0;
  const int P = fs.passes + (fs.compensate ? 1 : 0);
  for (int p = 0; p < P; p++) {
    const double al = p < fs.passes ? 0.5 : 0.5 * fs.passes + 1.0;
    const double be = 0.5 * (1.0 - al);
    double r[2 * 16 + 1] = {0.0};
    for (int j = 0; j < len; j++) { r[j] += be * k[j]; r[j + 1] += al * k[j]; r[j + 2] += be * k[j]; }
    len += 2;
    for (int j = 0; j < len; j++) k[j] = r[j];
  }
  FilterTaps<T> ft;
  ft.P = P; ft.s = fs.stride; ft.H = P * fs.stride;
  for (int j = 0; j < 2 * 16 + 1; j++) ft.c[j] = T(j < len ? k[j] : 0.0);
  return ft;
}

template <class T>
void launch_filter_fields(const GridP& g, const FieldPtrs<T>& f, const FilterSpec& fs, bool enabled, cudaStream_t s) {
  if (!enabled) return;
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  size_t sm = tile_smem(ft.H, sizeof(T));
  cudaFuncSetAttribute(k_filter_fields<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_filter_fields<T><<<grd, blk, sm, s>>>(g, f, ft);
}

template <class T>
void launch_ampere(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, const FilterSpec& fs, bool filter_on,
                   const double* ion_x, const double* ion_c, double ion_coef, cudaStream_t s) {
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  if (filter_on) {
    size_t sm = tile_smem(ft.H, sizeof(T));
    cudaFuncSetAttribute(k_ampere<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ampere<T, true><<<grd, blk, sm, s>>>(g, f, pt, ft, ion_x, ion_c, ion_coef);
  } else {
    size_t sm = tile_smem(0, sizeof(T));
    k_ampere<T, false><<<grd, blk, sm, s>>>(g, f, pt, ft, ion_x, ion_c, ion_coef);
  }
}

template void launch_faraday<float>(const GridP&, const FieldPtrs<float>&, const PmlTabs&, double, double, double,
                                    bool, cudaStream_t);
template void launch_faraday<double>(const GridP&, const FieldPtrs<double>&, const PmlTabs&, double, double, double,
                                     bool, cudaStream_t);
template void launch_filter_fields<float>(const GridP&, const FieldPtrs<float>&, const FilterSpec&, bool, cudaStream_t);
template void launch_filter_fields<double>(const GridP&, const FieldPtrs<double>&, const FilterSpec&, bool,
                                           cudaStream_t);
template void launch_ampere<float>(const GridP&, const FieldPtrs<float>&, const PmlTabs&, const FilterSpec&, bool,
                                   const double*, const double*, double, cudaStream_t);
template void launch_ampere<double>(const GridP&, const FieldPtrs<double>&, const PmlTabs&, const FilterSpec&, bool,
                                    const double*, const double*, double, cudaStream_t);

}  // namespace picgb
