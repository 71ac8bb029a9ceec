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

// ---------------------------------------------------------------------------
// TMA staging: one elected thread issues a 3D bulk tensor copy of the tile +
// halo (box BZ x BX x 1 of component c) into shared memory; completion is
// signalled on an mbarrier through the transaction byte count. Components are
// double-buffered, so the copy of component c+1 overlaps the filter of c.
// Waits are bounded: on timeout the kernel records ST_TIMEOUT, waits (bounded
// again) for its copies in flight and gives up the tile.
constexpr long kWaitLimit = 1L << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_box(void* dst, const CUtensorMap* map, int z, int x, int c, uint64_t* bar,
                                             uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"((unsigned long long)map), "r"(z), "r"(x), "r"(c), "r"(smem_u32(bar))
      : "memory");
}

// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (long it = 0; it < kWaitLimit; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

// A tiled bulk-tensor copy needs a 128-byte aligned shared destination: the
// staging buffers start at the dynamic shared base rounded up to 128 bytes and
// lie a whole number of 128-byte lines apart.
template <class T>
__host__ __device__ __forceinline__ int tile_stride(const TileMaps& tm) {
  const int line = 128 / (int)sizeof(T);
  return (tm.BX * tm.BZ + line - 1) / line * line;
}

__device__ __forceinline__ unsigned char* align128(unsigned char* p) {
  return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

// stage component c of a block into a shared buffer (leader thread only)
template <class T>
__device__ __forceinline__ void stage(T* buf, const CUtensorMap* map, int c, int gk0, int gi0, uint64_t* bar,
                                      const TileMaps& tm) {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tma_load_box(buf, map, gk0, gi0, c, bar, (uint32_t)(tm.BX * tm.BZ * sizeof(T)));
}

// x-pass: B1[ti][lk] = sum_j c_j A[ti + H + (j - P) s][lk + zoff] for the tile's rows
template <class T>
__device__ __forceinline__ void xpass(const T* A, T* B1, const FilterTaps<T>& ft, int BZ, int zoff, int WZ) {
  for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
    for (int lk = threadIdx.x; lk < WZ; lk += FT_Z) {
      const T* col = A + (ti + ft.H - ft.P * ft.s) * BZ + lk + zoff;
      T acc = T(0);
      for (int j = 0; j <= 2 * ft.P; j++) acc += ft.c[j] * col[j * ft.s * BZ];
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

__device__ __forceinline__ void tile_timeout(Ctrl* ctrl, uint64_t* bar0, uint64_t* bar1) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicOr(&ctrl->status, ST_TIMEOUT);
    // bounded: let any copy still in flight land before the block exits
    mbar_wait(bar0, 0); mbar_wait(bar0, 1);
    mbar_wait(bar1, 0); mbar_wait(bar1, 1);
  }
}

// gather copies: fE = F(E^n), fB = F(Bavg)
template <class T>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_filter_fields(GridP g, FieldPtrs<T> f, FilterTaps<T> ft,
                                                               const __grid_constant__ CUtensorMap mapE,
                                                               const __grid_constant__ CUtensorMap mapB, TileMaps tm,
                                                               Ctrl* ctrl) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* tile0 = reinterpret_cast<T*>(align128(smraw));
  T* tile1 = tile0 + tile_stride<T>(tm);
  const int H = ft.H;
  const int WZ = FT_Z + 2 * H;
  T* B1 = tile1 + tile_stride<T>(tm);
  __shared__ __align__(8) uint64_t bar[2];
  const int i0 = blockIdx.y * FT_X, k0 = blockIdx.x * FT_Z;
  const int gi0 = i0 - tm.H, gk0 = k0 - tm.HZ;
  const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
  if (leader) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (leader) stage<T>(tile0, &mapE, 0, gk0, gi0, &bar[0], tm);
  for (int c = 0; c < 6; c++) {
    T* A = (c & 1) ? tile1 : tile0;
    if (leader && c + 1 < 6)
      stage<T>((c & 1) ? tile0 : tile1, c + 1 < 3 ? &mapE : &mapB, (c + 1) % 3, gk0, gi0, &bar[(c + 1) & 1], tm);
    if (!mbar_wait(&bar[c & 1], (c >> 1) & 1)) {
      tile_timeout(ctrl, &bar[0], &bar[1]);
      return;
    }
    T* dst = c < 3 ? f.fE[c] : f.fB[c - 3];
    xpass<T>(A + (tm.H - H) * tm.BZ, B1, ft, tm.BZ, tm.HZ - H, WZ);
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
                                                        const double* ion_x, const double* ion_c, double ion_coef,
                                                        const __grid_constant__ CUtensorMap mapJ, TileMaps tm,
                                                        Ctrl* ctrl) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* tile0 = reinterpret_cast<T*>(align128(smraw));
  T* tile1 = tile0 + tile_stride<T>(tm);
  const int H = FILT ? ft.H : 0;
  const int WZ = FT_Z + 2 * H;
  T* B1 = tile1 + tile_stride<T>(tm);
  __shared__ __align__(8) uint64_t bar[2];
  const int i0 = blockIdx.y * FT_X, k0 = blockIdx.x * FT_Z;
  const int gi0 = i0 - tm.H, gk0 = k0 - tm.HZ;
  const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
  if (leader) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (leader) stage<T>(tile0, &mapJ, 0, gk0, gi0, &bar[0], tm);
  const T dt = T(g.dt);
  const T c2 = T(kC * kC);
  const T ie0 = T(1.0 / kEps0);
  const double c2d = kC * kC;
  const int k = k0 + threadIdx.x;
  for (int c = 0; c < 3; c++) {
    T* A = (c & 1) ? tile1 : tile0;
    if (leader && c + 1 < 3) stage<T>((c & 1) ? tile0 : tile1, &mapJ, c + 1, gk0, gi0, &bar[(c + 1) & 1], tm);
    if (!mbar_wait(&bar[c & 1], (c >> 1) & 1)) {
      tile_timeout(ctrl, &bar[0], &bar[1]);
      return;
    }
    if (c == 2 && ion_x != nullptr) {
      // rigid ion-column current added to Jz before the filter
      for (int li = threadIdx.y; li < tm.BX; li += FT_TY) {
        const int gi = gi0 + li;
        if (gi < 0 || gi > g.nx) continue;
        const double ix = ion_coef * ion_x[gi];
        for (int lk = threadIdx.x; lk < tm.BZ; lk += FT_Z) {
          const int gk = gk0 + lk;
          if (gk >= 0 && gk <= g.nz) A[li * tm.BZ + lk] += T(ix * ion_c[gk]);
        }
      }
      __syncthreads();
    }
    int vi0, vi1, vk0, vk1;
    valid_range(c, g.nx, g.nz, vi0, vi1, vk0, vk1);
    if (FILT) {
      xpass<T>(A + (tm.H - H) * tm.BZ, B1, ft, tm.BZ, tm.HZ - H, WZ);
      __syncthreads();
    }
    for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
      const int i = i0 + ti;
      if (i > g.nx || k > g.nz) continue;
      const long p = (long)i * g.ld + k;
      f.Jn[c][p] = T(0);
      const bool v = i >= vi0 && i <= vi1 && k >= vk0 && k <= vk1;
      if (!v) {
        f.Eo[c][p] = T(0);
        continue;
      }
      const T jv = FILT ? zpass<T>(B1, ft, WZ, ti, threadIdx.x) : A[(ti + tm.H) * tm.BZ + threadIdx.x + tm.HZ];
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

template <class T>
static size_t tile_smem(const TileMaps& tm, int H) {
  // + 128: room to round the dynamic shared base up to a 128-byte line
  return (2 * (size_t)tile_stride<T>(tm) + (size_t)FT_X * (FT_Z + 2 * H)) * sizeof(T) + 128;
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
    for (int j = 0; j < len; j++) {
      r[j] += be * k[j];
      r[j + 1] += al * k[j];
      r[j + 2] += be * k[j];
    }
    len += 2;
    for (int j = 0; j < len; j++) k[j] = r[j];
  }
  FilterTaps<T> ft;
  ft.P = P;
  ft.s = fs.stride;
  ft.H = P * fs.stride;
  for (int j = 0; j < 2 * 16 + 1; j++) ft.c[j] = T(j < len ? k[j] : 0.0);
  return ft;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// 3D tensor over a 3-component block: (nz+1) x (nx+1) x 3, rows ld elements apart, components cs apart
template <class T>
static bool encode_block(CUtensorMap* m, const void* base, const GridP& g, const TileMaps& tm) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)(g.nz + 1), (cuuint64_t)(g.nx + 1), 3};
  const cuuint64_t strides[2] = {(cuuint64_t)g.ld * sizeof(T), (cuuint64_t)g.cs * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)tm.BZ, (cuuint32_t)tm.BX, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  return fn(m, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

template <class T>
bool make_tile_maps(const GridP& g, const FieldPtrs<T>& f, int H, TileMaps& tm) {
  // a box starts at z = k0 - HZ, which must be 16-byte aligned: k0 is a multiple of 64 and HZ of 4
  tm.H = H;
  tm.HZ = (H + 3) & ~3;
  tm.BX = FT_X + 2 * H;
  tm.BZ = FT_Z + 2 * tm.HZ;
  tm.ok = false;
  if (tm.BX > 256 || tm.BZ > 256) return false;
  if (tile_smem<T>(tm, H) > 227 * 1024) return false;
  tm.Ebase[0] = f.E[0];
  tm.Ebase[1] = f.Eo[0];
  tm.Jbase[0] = f.J[0];
  tm.Jbase[1] = f.Jn[0];
  const bool ok = encode_block<T>(&tm.E[0], f.E[0], g, tm) && encode_block<T>(&tm.E[1], f.Eo[0], g, tm) &&
                  encode_block<T>(&tm.J[0], f.J[0], g, tm) && encode_block<T>(&tm.J[1], f.Jn[0], g, tm) &&
                  encode_block<T>(&tm.Bavg, f.Bavg[0], g, tm);
  tm.ok = ok;
  return ok;
}

template <class T>
void launch_filter_fields(const GridP& g, const FieldPtrs<T>& f, const FilterSpec& fs, bool enabled,
                          const TileMaps& tm, Ctrl* ctrl, cudaStream_t s) {
  if (!enabled) return;
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  const size_t sm = tile_smem<T>(tm, ft.H);
  const CUtensorMap& mE = tm.Ebase[0] == (const void*)f.E[0] ? tm.E[0] : tm.E[1];
  cudaFuncSetAttribute(k_filter_fields<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_filter_fields<T><<<grd, blk, sm, s>>>(g, f, ft, mE, tm.Bavg, tm, ctrl);
}

template <class T>
void launch_ampere(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, const FilterSpec& fs, bool filter_on,
                   const double* ion_x, const double* ion_c, double ion_coef, const TileMaps& tm, Ctrl* ctrl,
                   cudaStream_t s) {
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  const CUtensorMap& mJ = tm.Jbase[0] == (const void*)f.J[0] ? tm.J[0] : tm.J[1];
  const size_t sm = tile_smem<T>(tm, filter_on ? ft.H : 0);
  if (filter_on) {
    cudaFuncSetAttribute(k_ampere<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ampere<T, true><<<grd, blk, sm, s>>>(g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl);
  } else {
    cudaFuncSetAttribute(k_ampere<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_ampere<T, false><<<grd, blk, sm, s>>>(g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl);
  }
}

template void launch_faraday<float>(const GridP&, const FieldPtrs<float>&, const PmlTabs&, double, double, double,
                                    bool, cudaStream_t);
template void launch_faraday<double>(const GridP&, const FieldPtrs<double>&, const PmlTabs&, double, double, double,
                                     bool, cudaStream_t);
#define INSTF(T)                                                                                                 \
  template bool make_tile_maps<T>(const GridP&, const FieldPtrs<T>&, int, TileMaps&);                            \
  template void launch_filter_fields<T>(const GridP&, const FieldPtrs<T>&, const FilterSpec&, bool, const TileMaps&, \
                                        Ctrl*, cudaStream_t);                                                    \
  template void launch_ampere<T>(const GridP&, const FieldPtrs<T>&, const PmlTabs&, const FilterSpec&, bool,       \
                                 const double*, const double*, double, const TileMaps&, Ctrl*, cudaStream_t);
INSTF(float)
INSTF(double)
#undef INSTF

}  // namespace picgb
