// Field kernels of the boosted-frame PIC step:
//  - Faraday with the tunable (Cole-Karkkainen) operator, Friedman damping and
//    the split-field PML for B (Eq. Faraday, Eq. Faraday_Friedman, App. II);
//  - the multi-pass bilinear filter with compensation (Sec. 4.1), applied to
//    the fields used by the gather, tile by tile in shared memory;
//  - Ampere with the Yee operator and the split-field PML for E, fused with the
//    filter of the deposited current and the rigid ion-column current.
#include <type_traits>

#include "pic_common.cuh"

namespace picgb {

namespace {


constexpr int FT_X = 16;
constexpr int FT_Z = 64;
constexpr int FT_TY = 4;

// B^{n-1/2} of the thread's rows of a tile (rows ty, ty + FT_TY, ...; column k0 + tx), loaded together so
// that their latencies overlap (and, in the fused kernel, overlap the tile's bulk copies)
template <class T>
struct TileB {
  static constexpr int NR = FT_X / FT_TY;
  T x[NR], y[NR], z[NR];
};

template <class T>
__device__ __forceinline__ void load_tile_b(const GridP& g, const FieldPtrs<T>& f, int i0, int k0, TileB<T>& b) {
  const int k = k0 + threadIdx.x;
#pragma unroll
  for (int r = 0; r < TileB<T>::NR; r++) {
    const int i = i0 + threadIdx.y + r * FT_TY;
    const long p = (long)i * g.ld + k;
    const bool in = i <= g.nx && k <= g.nz;
    b.x[r] = (in && k <= g.nz - 1) ? f.B[0][p] : T(0);
    b.z[r] = (in && i <= g.nx - 1) ? f.B[2][p] : T(0);
    b.y[r] = (in && i <= g.nx - 1 && k <= g.nz - 1) ? f.B[1][p] : T(0);
  }
}

// B update of one tile from E_eff staged in shared memory: Ee[c] holds the tile and a one-node halo, row
// stride SZ, node (i0 - 1 + li, k0 - 1 + lk) at li * SZ + lk (zero outside the grid); b: the tile's
// B^{n-1/2} (load_tile_b). PML = false: a tile clear of the PML (no table reads, no FP64 in the
// instruction stream)
template <class T, bool CK, bool PML>
__device__ __forceinline__ void faraday_update_t(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt,
                                                 const FarK<T>& q, const T* const* Ee, const int SZ, int i0,
                                                 int k0, const TileB<T>& b) {
  constexpr bool interior = !PML;
  const T dt = grid_dt<T>(g), idx = grid_idx<T>(g), idz = grid_idz<T>(g);
  const int k = k0 + threadIdx.x;
  constexpr int NR = TileB<T>::NR;
  const T* bx0 = b.x;
  const T* by0 = b.y;
  const T* bz0 = b.z;
#pragma unroll
  for (int r = 0; r < NR; r++) {
    const int ti = threadIdx.y + r * FT_TY;
    const int i = i0 + ti;
    if (i > g.nx || k > g.nz) continue;
    const long p = (long)i * g.ld + k;
    const int s0 = (ti + 1) * SZ + threadIdx.x + 1;   // node (i, k) in the staged tile
    // Delta*_z at (i, k+1/2) and Delta*_x at (i+1/2, k) of component c
    auto dsz = [&](int c) {
      const T* E = Ee[c];
      const T d0 = E[s0 + 1] - E[s0];
      if (!CK) return d0 * idz;
      const T dp = E[s0 + SZ + 1] - E[s0 + SZ];
      const T dm = E[s0 - SZ + 1] - E[s0 - SZ];
      return (q.a2 * d0 + q.b2 * (dp + dm)) * idz;
    };
    auto dsx = [&](int c) {
      const T* E = Ee[c];
      const T d0 = E[s0 + SZ] - E[s0];
      if (!CK) return d0 * idx;
      const T dp = E[s0 + SZ + 1] - E[s0 + 1];
      const T dm = E[s0 + SZ - 1] - E[s0 - 1];
      return (q.a2 * d0 + q.b2 * (dp + dm)) * idx;
    };
    // Bx at (i, k+1/2): dBx/dt = Delta*_z Ey
    if (k <= g.nz - 1) {
      const T d = dsz(EY);
      const T bo = bx0[r];
      T bn;
      if (!interior && pt.sz_h[k] > 0.0) bn = T(pt.xz_h[k] * (double)bo + pt.cz_h[k] * (double)d);
      else bn = bo + dt * d;
      f.B[0][p] = bn;
      f.Bavg[0][p] = T(0.5) * (bo + bn);
    }
    // Bz at (i+1/2, k): dBz/dt = -Delta*_x Ey
    if (i <= g.nx - 1) {
      const T d = dsx(EY);
      const T bo = bz0[r];
      T bn;
      if (!interior && pt.sx_h[i] > 0.0) bn = T(pt.xx_h[i] * (double)bo - pt.cx_h[i] * (double)d);
      else bn = bo - dt * d;
      f.B[2][p] = bn;
      f.Bavg[2][p] = T(0.5) * (bo + bn);
    }
    // By at (i+1/2, k+1/2): dBy/dt = -Delta*_z Ex + Delta*_x Ez; split in the PML
    if (i <= g.nx - 1 && k <= g.nz - 1) {
      const T a = dsz(EX);
      const T b = dsx(EZ);
      const T bo = by0[r];
      T bn;
      if (!interior && (pt.sx_h[i] > 0.0 || pt.sz_h[k] > 0.0)) {
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
  }
}


template <class T, bool CK>
__device__ __forceinline__ void faraday_update(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt,
                                               const FarK<T>& q, const T* const* Ee, const int SZ, int i0,
                                               int k0, const TileB<T>& b) {
  // block-uniform: the tiles clear of the PML take the instantiation without its branches
  const bool interior = i0 >= pt.iin0 && i0 + FT_X - 1 <= pt.iin1 && k0 >= pt.kin0 && k0 + FT_Z - 1 <= pt.kin1;
  if (interior) faraday_update_t<T, CK, false>(g, f, pt, q, Ee, SZ, i0, k0, b);
  else faraday_update_t<T, CK, true>(g, f, pt, q, Ee, SZ, i0, k0, b);
}

// Faraday + PML-B over a tile of FT_X x FT_Z nodes (threads FT_Z x FT_TY). The
// Friedman field E_eff (Eq. 7) of the tile's nodes and a one-node halo is built
// once in shared memory (zero outside the grid); the Friedman average update
// is written from the same loads. Delta*_z, Delta*_x are the CK operators
// reduced to 2D (PR-2, PR-3). Tiles clear of the PML take the plain update.
template <class T, bool FRIED, bool CK>
__device__ __forceinline__ void faraday_tile(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt,
                                             const FarK<T>& q, int tile_k, int tile_i) {
  constexpr int SX = FT_X + 2, SZ = FT_Z + 2;
  __shared__ T Ee[3][SX * SZ];
  const int i0 = tile_i * FT_X, k0 = tile_k * FT_Z;
  TileB<T> bold;
  load_tile_b<T>(g, f, i0, k0, bold);
  const int tid = threadIdx.y * FT_Z + threadIdx.x;
  for (int e = tid; e < SX * SZ; e += FT_Z * FT_TY) {
    const int li = e / SZ, lk = e - li * SZ;
    const int i = i0 - 1 + li, k = k0 - 1 + lk;
    const bool in = i >= 0 && i <= g.nx && k >= 0 && k <= g.nz;
    const bool own = in && li >= 1 && li <= FT_X && lk >= 1 && lk <= FT_Z;
    const long p = (long)i * g.ld + k;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      T v = T(0);
      if (in) {
        const T en = f.E[c][p];
        if (FRIED) {
          const T eb = f.Eb[c][p];
          v = q.c1 * en + q.c2 * f.Eo[c][p] + q.c3 * eb;
          if (own) f.Ebn[c][p] = q.h1 * en + q.h2 * eb;
        } else {
          v = en;
        }
      }
      Ee[c][e] = v;
    }
  }
  __syncthreads();
  const T* Eep[3] = {Ee[0], Ee[1], Ee[2]};
  faraday_update<T, CK>(g, f, pt, q, Eep, SZ, i0, k0, bold);
}

template <class T, bool FRIED, bool CK>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_faraday(GridP g, FieldPtrs<T> f, PmlTabs pt, FarK<T> q) {
  faraday_tile<T, FRIED, CK>(g, f, pt, q, blockIdx.x, blockIdx.y);
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

// a box copy counted by an expect_tx issued beforehand
__device__ __forceinline__ void tma_copy_box(void* dst, const CUtensorMap* map, int z, int x, int c, uint64_t* bar) {
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

// the fused Faraday kernel's boxes of E^{n-1} and E-bar: FT_X + 2 rows by FT_Z + 8 columns, whole lines
template <class T>
__host__ __device__ constexpr int ring_stride() {
  return ((FT_X + 2) * (FT_Z + 8) + 128 / (int)sizeof(T) - 1) / (128 / (int)sizeof(T)) * (128 / (int)sizeof(T));
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

// Composed filter over a staged tile: the x-pass writes B1 (FT_X rows of the
// tile, WZ = FT_Z + 2H columns, row stride WZP), the z-pass writes Zb (FT_X x
// FT_Z). A points at the element (tile row -H, tile column -H) of the staged
// box, whose row stride is BZ.
static_assert(FT_X == 16 && FT_TY == 4 && FT_Z == 64, "filter blocking assumes 16 x 64 tiles and 64 x 4 threads");

__host__ __device__ constexpr int filter_wzp(int H) { return (FT_Z + 2 * H + 3) / 4 * 4; }

// any number of passes and any stride (runtime tap loops)
template <class T>
__device__ __forceinline__ void filter_tile_any(const T* A, int BZ, T* B1, T* Zb, const FilterTaps<T>& ft) {
  const int WZ = FT_Z + 2 * ft.H, WZP = filter_wzp(ft.H);
  for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
    for (int lk = threadIdx.x; lk < WZ; lk += FT_Z) {
      const T* col = A + (ti + ft.H - ft.P * ft.s) * BZ + lk;
      T acc = T(0);
      for (int j = 0; j <= 2 * ft.P; j++) acc += ft.c[j] * col[j * ft.s * BZ];
      B1[ti * WZP + lk] = acc;
    }
  }
  __syncthreads();
  for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
    const T* row = B1 + ti * WZP + threadIdx.x + ft.H - ft.P * ft.s;
    T acc = T(0);
    for (int j = 0; j <= 2 * ft.P; j++) acc += ft.c[j] * row[j * ft.s];
    Zb[ti * FT_Z + threadIdx.x] = acc;
  }
  __syncthreads();
}

// P passes at stride 1 with the taps unrolled: each thread filters four
// consecutive values from a register window of 4 + 2P inputs (x-pass: four rows
// of one column; z-pass: four columns of one row, read as 16-byte vectors). The
// FP32 path takes filter_tile_fixed_f32 (below); this form serves FP64.
template <class T>
struct Vec16;
template <>
struct Vec16<double> { typedef double2 type; static constexpr int n = 2; };

// FP32: the x-pass works on pairs of columns with packed FMAs (one 8-byte load and one FFMA2 serve two
// columns). A pair must start at an even element both in the staged box and in B1; where the box's
// first filter column is odd ((HZ - H) odd, HZ = H rounded up to 4), B1 carries one leading pad column
// and the z-pass reads its window one element early.
// With STORE the z-pass writes its four outputs straight to dst (row i0 + ti, columns k0 + g4 ...; a
// 16-byte store where all four lie inside the grid) instead of to Zb.
template <int P, bool STORE = false>
__device__ __forceinline__ void filter_tile_fixed_f32(const float* A, int BZ, float* B1, float* Zb,
                                                      const FilterTaps<float>& ft, float* dst = nullptr,
                                                      const GridP* g = nullptr, int i0 = 0, int k0 = 0) {
  constexpr int NT = 2 * P + 1, NW = 4 + 2 * P;
  constexpr int WZ = FT_Z + 2 * P, WZP = filter_wzp(P);
  constexpr int HZ = (P + 3) & ~3, PAD = (HZ - P) & 1;
  constexpr int NPAIR = (WZ + PAD + 1) / 2;
  static_assert(2 * NPAIR <= WZP, "B1 row holds the pad and every pair");
  // the staged box's row stride as a constant (a stride-1 filter of P passes has halo P, and the tile maps'
  // boxes are FT_Z + 2 HZ wide): every load below addresses with an immediate offset
  constexpr int BZC = FT_Z + 2 * HZ;
  (void)BZ;
  const int tid = threadIdx.y * FT_Z + threadIdx.x;
  for (int task = tid; task < (FT_X / 4) * NPAIR; task += FT_Z * FT_TY) {
    const int rq = task / NPAIR, cpair = task - rq * NPAIR;
    const int r0 = 4 * rq, b = 2 * cpair;   // B1 column b <-> filter column b - PAD
    const float* col = A + r0 * BZC + b - PAD;
    float2 v[NW];
#pragma unroll
    for (int j = 0; j < NW; j++) v[j] = *reinterpret_cast<const float2*>(col + j * BZC);
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < NT; j++) acc = __ffma2_rn(make_float2(ft.c[j], ft.c[j]), v[q + j], acc);
      *reinterpret_cast<float2*>(B1 + (r0 + q) * WZP + b) = acc;
    }
  }
  __syncthreads();
  {
    constexpr int NV = (NW + PAD + 3) / 4;   // float4 vectors covering the pad and the window
    const int ti = tid >> 4, g4 = (tid & 15) * 4;
    float v[NV * 4];
    const float4* row = reinterpret_cast<const float4*>(B1 + ti * WZP + g4);
#pragma unroll
    for (int u = 0; u < NV; u++) {
      const float4 x = row[u];
      v[4 * u] = x.x; v[4 * u + 1] = x.y; v[4 * u + 2] = x.z; v[4 * u + 3] = x.w;
    }
    float o[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < NT; j++) acc = fmaf(ft.c[j], v[PAD + q + j], acc);
      o[q] = acc;
    }
    if constexpr (STORE) {
      const int gi = i0 + ti, gk = k0 + g4;
      if (gi <= g->nx) {
        float* d = dst + (long)gi * g->ld + gk;
        if (gk + 3 <= g->nz) {
          *reinterpret_cast<float4*>(d) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; q++)
            if (gk + q <= g->nz) d[q] = o[q];
        }
      }
    } else {
      *reinterpret_cast<float4*>(Zb + ti * FT_Z + g4) = make_float4(o[0], o[1], o[2], o[3]);
    }
  }
  __syncthreads();
}

template <class T, int P>
__device__ __forceinline__ void filter_tile_fixed(const T* A, int BZ, T* B1, T* Zb, const FilterTaps<T>& ft) {
  constexpr int NT = 2 * P + 1, NW = 4 + 2 * P;
  constexpr int WZ = FT_Z + 2 * P, WZP = filter_wzp(P);
  {
    const int r0 = 4 * threadIdx.y;
    for (int lk = threadIdx.x; lk < WZ; lk += FT_Z) {
      T v[NW];
#pragma unroll
      for (int j = 0; j < NW; j++) v[j] = A[(r0 + j) * BZ + lk];
#pragma unroll
      for (int q = 0; q < 4; q++) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; j < NT; j++) acc += ft.c[j] * v[q + j];
        B1[(r0 + q) * WZP + lk] = acc;
      }
    }
  }
  __syncthreads();
  {
    typedef typename Vec16<T>::type V;
    constexpr int VN = Vec16<T>::n;
    constexpr int NV = (NW + VN - 1) / VN;   // vectors covering the window (stays inside the row)
    const int tid = threadIdx.y * FT_Z + threadIdx.x;
    const int ti = tid >> 4, g4 = (tid & 15) * 4;
    T v[NV * VN];
    const V* row = reinterpret_cast<const V*>(B1 + ti * WZP + g4);
#pragma unroll
    for (int u = 0; u < NV; u++) {
      const V x = row[u];
      if constexpr (VN == 4) {
        v[4 * u] = x.x; v[4 * u + 1] = x.y; v[4 * u + 2] = x.z; v[4 * u + 3] = x.w;
      } else {
        v[2 * u] = x.x; v[2 * u + 1] = x.y;
      }
    }
    T o[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      T acc = T(0);
#pragma unroll
      for (int j = 0; j < NT; j++) acc += ft.c[j] * v[q + j];
      o[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < 4; q++) Zb[ti * FT_Z + g4 + q] = o[q];
  }
  __syncthreads();
}

template <class T, int PT>
__device__ __forceinline__ void filter_tile(const T* A, int BZ, T* B1, T* Zb, const FilterTaps<T>& ft) {
  if constexpr (PT > 0 && sizeof(T) == 4) filter_tile_fixed_f32<PT>(A, BZ, B1, Zb, ft);
  else if constexpr (PT > 0) filter_tile_fixed<T, PT>(A, BZ, B1, Zb, ft);
  else filter_tile_any<T>(A, BZ, B1, Zb, ft);
}

// the filtered tile written to dst (the tile's nodes inside the grid)
template <class T, int PT>
__device__ __forceinline__ void filter_tile_to(const T* A, int BZ, T* B1, T* Zb, const FilterTaps<T>& ft, T* dst,
                                               const GridP& g, int i0, int k0) {
  if constexpr (PT > 0 && sizeof(T) == 4) {
    filter_tile_fixed_f32<PT, true>(A, BZ, B1, Zb, ft, dst, &g, i0, k0);
  } else {
    filter_tile<T, PT>(A, BZ, B1, Zb, ft);
    const int gk = k0 + threadIdx.x;
    for (int ti = threadIdx.y; ti < FT_X; ti += FT_TY) {
      const int gi = i0 + ti;
      if (gi <= g.nx && gk <= g.nz) dst[(long)gi * g.ld + gk] = Zb[ti * FT_Z + threadIdx.x];
    }
  }
}

// Block-wide wait for a staged copy: one warp polls the mbarrier (the other warps wait at the barrier
// instruction, which takes no issue slots from the SM's other blocks); the bar.sync that follows orders
// the copy's arrival before every thread's reads. Returns false, block-uniformly, on timeout.
__device__ __forceinline__ bool block_wait(uint64_t* bar, uint32_t parity) {
  bool ok = true;
  if (threadIdx.y == 0 && threadIdx.x < 32) ok = mbar_wait(bar, parity);
  return __syncthreads_or(!ok) == 0;
}

__device__ __forceinline__ void tile_timeout(Ctrl* ctrl, uint64_t* bar0, uint64_t* bar1) {
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    atomicOr(&ctrl->status, ST_TIMEOUT);
    // bounded: let any copy still in flight land before the block exits
    mbar_wait(bar0, 0); mbar_wait(bar0, 1);
    mbar_wait(bar1, 0); mbar_wait(bar1, 1);
  }
}

// gather copies: fE = F(E^n), fB = F(Bavg). PT > 0: PT passes at stride 1.
template <class T, int PT>
__device__ __forceinline__ void filter_fields_tile(const GridP& g, const FieldPtrs<T>& f, const FilterTaps<T>& ft,
                                                   const CUtensorMap* pmapE, const CUtensorMap* pmapB,
                                                   const TileMaps& tm, Ctrl* ctrl, int tile_k, int tile_i,
                                                   int c_first = 0) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* tile0 = reinterpret_cast<T*>(align128(smraw));
  T* tile1 = tile0 + tile_stride<T>(tm);
  const int H = ft.H;
  T* B1 = tile1 + tile_stride<T>(tm);
  T* Zb = B1 + FT_X * filter_wzp(H);
  __shared__ __align__(8) uint64_t bar[2];
  const int i0 = tile_i * FT_X, k0 = tile_k * FT_Z;
  const int gi0 = i0 - tm.H, gk0 = k0 - tm.HZ;
  const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
  if (leader) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (leader) stage<T>(tile0, c_first < 3 ? pmapE : pmapB, c_first % 3, gk0, gi0, &bar[0], tm);
  for (int c = c_first; c < 6; c++) {
    const int u = c - c_first;   // staging slot and phase follow the components handled
    T* A = (u & 1) ? tile1 : tile0;
    if (leader && c + 1 < 6)
      stage<T>((u & 1) ? tile0 : tile1, c + 1 < 3 ? pmapE : pmapB, (c + 1) % 3, gk0, gi0, &bar[(u + 1) & 1], tm);
    if (!block_wait(&bar[u & 1], (u >> 1) & 1)) {
      tile_timeout(ctrl, &bar[0], &bar[1]);
      return;
    }
    T* dst = c < 3 ? f.fE[c] : f.fB[c - 3];
    filter_tile_to<T, PT>(A + (tm.H - H) * tm.BZ + (tm.HZ - H), tm.BZ, B1, Zb, ft, dst, g, i0, k0);
    // Zb and the other staging buffer are rewritten only after the next filter_tile's first barrier
  }
}

template <class T, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_filter_fields(GridP g, FieldPtrs<T> f, FilterTaps<T> ft,
                                                               const __grid_constant__ CUtensorMap mapE,
                                                               const __grid_constant__ CUtensorMap mapB, TileMaps tm,
                                                               Ctrl* ctrl, int c_first) {
  filter_fields_tile<T, PT>(g, f, ft, &mapE, &mapB, tm, ctrl, blockIdx.x, blockIdx.y, c_first);
}

// Faraday with its E tiles staged by TMA, fused with the gather filter of E^n. One round of bulk tensor
// copies brings the tile's E^n with the filter's halo (serving both the Friedman field and the filter)
// and, under Friedman damping, E^{n-1} and E-bar on the tile and a one-node halo (boxes of FT_X + 2 rows
// by FT_Z + 8 columns, starting 16-byte aligned at k0 - 4). E_eff (Eq. 7) is formed in place of the
// staged E^{n-1}; B, B_avg and E-bar are updated as in k_faraday, then F(E^n) is written for the gather
// (k_filter_fields then filters B_avg only).
template <class T, bool FRIED, bool CK, int PT>
__device__ __forceinline__ void faraday_fused_tile(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt,
                                                   const FarK<T>& q, const FilterTaps<T>& ft,
                                                   const CUtensorMap* mapE, const CUtensorMap* mapEo,
                                                   const CUtensorMap* mapEb, Ctrl* ctrl, int tile_k, int tile_i) {
  constexpr int SX = FT_X + 2, SZ = FT_Z + 2, RZ = FT_Z + 8;
  // the staged boxes' geometry as constants: a stride-1 filter of PT passes has halo H = PT (the host
  // checks that the tile maps were built for it), the boxes are FT_X + 2 H rows of FT_Z + 2 HZ
  constexpr int H = PT, HZ = (PT + 3) & ~3, BX = FT_X + 2 * H, BZ = FT_Z + 2 * HZ;
  constexpr int LINE = 128 / (int)sizeof(T), stride = (BX * BZ + LINE - 1) / LINE * LINE;
  extern __shared__ __align__(128) unsigned char smraw[];
  const int rstride = ring_stride<T>();
  T* A = reinterpret_cast<T*>(align128(smraw));   // E^n, three boxes with the filter halo
  T* R = A + 3 * stride;                          // E^{n-1} then E-bar, three components each (FRIED)
  // the filter's scratch reuses R once the B update has read E_eff (four CTAs fit on an SM)
  T* B1 = R;
  T* Zb = B1 + FT_X * filter_wzp(H);
  __shared__ __align__(8) uint64_t bar[1];
  const int i0 = tile_i * FT_X, k0 = tile_k * FT_Z;
  const int gi0 = i0 - H, gk0 = k0 - HZ;
  const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
  if (leader) {
    mbar_init(&bar[0]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (leader) {
    const uint32_t box = (uint32_t)(BX * BZ * sizeof(T)), rbox = (uint32_t)(SX * RZ * sizeof(T));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(&bar[0])),
                 "r"(3 * box + (FRIED ? 6 * rbox : 0u))
                 : "memory");
    for (int c = 0; c < 3; c++) tma_copy_box(A + c * stride, mapE, gk0, gi0, c, &bar[0]);
    if (FRIED)
      for (int c = 0; c < 3; c++) {
        tma_copy_box(R + c * rstride, mapEo, k0 - 4, i0 - 1, c, &bar[0]);
        tma_copy_box(R + (3 + c) * rstride, mapEb, k0 - 4, i0 - 1, c, &bar[0]);
      }
  }
  // the tile's B^{n-1/2} in flight while the copies land
  TileB<T> bold;
  load_tile_b<T>(g, f, i0, k0, bold);
  // the wait's outcome is made block-uniform, so that no thread is left at a later barrier
  if (!block_wait(&bar[0], 0)) {
    tile_timeout(ctrl, &bar[0], &bar[0]);
    return;
  }
  const T* Eep[3];
  int esz;
  if (FRIED) {
    // E_eff = c1 E^n + c2 E^{n-1} + c3 E-bar on the tile and its halo, in place of E^{n-1}; E-bar's update
    // for the tile's own nodes
    constexpr int off = (H - 1) * BZ + (HZ - 1);   // box element of node (i0 - 1, k0 - 1)
    // E-bar's update of the tile's own nodes first (read before E_eff overwrites nothing it needs: E_eff
    // replaces E^{n-1}, E-bar's box is only read)
    const int k = k0 + threadIdx.x;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const T* Ac = A + c * stride + off + BZ + 1;
      const T* Rb = R + (3 + c) * rstride + RZ + 4;
#pragma unroll
      for (int r = 0; r < FT_X / FT_TY; r++) {
        const int ti = threadIdx.y + r * FT_TY, i = i0 + ti;
        if (i <= g.nx && k <= g.nz)
          f.Ebn[c][(long)i * g.ld + k] = q.h1 * Ac[ti * BZ + threadIdx.x] + q.h2 * Rb[ti * RZ + threadIdx.x];
      }
    }
    // rows ty, ty + 4, ... of the tile + halo, columns tx and (two threads) tx + FT_Z: unrolled with
    // constant strides
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const T* Ac = A + c * stride + off + threadIdx.y * BZ + threadIdx.x;
      T* Ro = R + c * rstride + 3 + threadIdx.y * RZ + threadIdx.x;
      const T* Rb = R + (3 + c) * rstride + 3 + threadIdx.y * RZ + threadIdx.x;
#pragma unroll
      for (int m = 0; m < (SX + FT_TY - 1) / FT_TY; m++) {
        if (threadIdx.y + m * FT_TY < SX) {
          Ro[m * FT_TY * RZ] = q.c1 * Ac[m * FT_TY * BZ] + q.c2 * Ro[m * FT_TY * RZ] + q.c3 * Rb[m * FT_TY * RZ];
          if (threadIdx.x < SZ - FT_Z)
            Ro[m * FT_TY * RZ + FT_Z] =
                q.c1 * Ac[m * FT_TY * BZ + FT_Z] + q.c2 * Ro[m * FT_TY * RZ + FT_Z] + q.c3 * Rb[m * FT_TY * RZ + FT_Z];
        }
      }
    }
    Eep[0] = R + 3;
    Eep[1] = R + rstride + 3;
    Eep[2] = R + 2 * rstride + 3;
    esz = RZ;
    __syncthreads();
  } else {
    for (int c = 0; c < 3; c++) Eep[c] = A + c * stride + (H - 1) * BZ + (HZ - 1);
    esz = BZ;
  }
  faraday_update<T, CK>(g, f, pt, q, Eep, esz, i0, k0, bold);
  // the gather copies of E^n: the filter of the staged boxes (its scratch overwrites E_eff: every thread's
  // B update has read it first)
  __syncthreads();
  for (int c = 0; c < 3; c++)
    filter_tile_to<T, PT>(A + c * stride + (HZ - H), BZ, B1, Zb, ft, f.fE[c], g, i0, k0);
}

template <class T, bool FRIED, bool CK, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY, 4) k_faraday_fused(GridP g, FieldPtrs<T> f, PmlTabs pt, FarK<T> q,
                                                               FilterTaps<T> ft,
                                                               const __grid_constant__ CUtensorMap mapE,
                                                               const __grid_constant__ CUtensorMap mapEo,
                                                               const __grid_constant__ CUtensorMap mapEb,
                                                               Ctrl* ctrl) {
  faraday_fused_tile<T, FRIED, CK, PT>(g, f, pt, q, ft, &mapE, &mapEo, &mapEb, ctrl, blockIdx.x, blockIdx.y);
}

// Ampere + PML-E, with the current (plus the ion column current) filtered in the tile first
template <class T, bool FILT, int PT>
__device__ __forceinline__ void ampere_tile(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt,
                                            const FilterTaps<T>& ft, const double* ion_x, const double* ion_c,
                                            double ion_coef, const CUtensorMap* pmapJ, const TileMaps& tm,
                                            Ctrl* ctrl, int tile_k, int tile_i) {
  extern __shared__ __align__(128) unsigned char smraw[];
  T* tile0 = reinterpret_cast<T*>(align128(smraw));
  T* tile1 = tile0 + tile_stride<T>(tm);
  const int H = FILT ? ft.H : 0;
  T* B1 = tile1 + tile_stride<T>(tm);
  T* Zb = B1 + FT_X * filter_wzp(H);
  __shared__ __align__(8) uint64_t bar[2];
  const int i0 = tile_i * FT_X, k0 = tile_k * FT_Z;
  const int gi0 = i0 - tm.H, gk0 = k0 - tm.HZ;
  const bool leader = threadIdx.x == 0 && threadIdx.y == 0;
  if (leader) {
    mbar_init(&bar[0]);
    mbar_init(&bar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (leader) stage<T>(tile0, pmapJ, 0, gk0, gi0, &bar[0], tm);
  const T dt = grid_dt<T>(g);
  const T c2 = T(kC * kC);
  const T ie0 = T(1.0 / kEps0);
  const T idx = grid_idx<T>(g), idz = grid_idz<T>(g);
  const double c2d = kC * kC;
  const int k = k0 + threadIdx.x;
  for (int c = 0; c < 3; c++) {
    T* A = (c & 1) ? tile1 : tile0;
    if (leader && c + 1 < 3) stage<T>((c & 1) ? tile0 : tile1, pmapJ, c + 1, gk0, gi0, &bar[(c + 1) & 1], tm);
    int vi0, vi1, vk0, vk1;
    valid_range(c, g.nx, g.nz, vi0, vi1, vk0, vk1);
    // E^n and the B^{n+1/2} values of the curl for the thread's rows, loaded before the wait for the
    // staged current and the filter, so that their latency overlaps both
    constexpr int NR = FT_X / FT_TY;
    T e0[NR], ba[NR], bb[NR], bc[NR], bd[NR];
#pragma unroll
    for (int r = 0; r < NR; r++) {
      const int i = i0 + threadIdx.y + r * FT_TY;
      const long p = (long)i * g.ld + k;
      const bool v = i <= g.nx && k <= g.nz && i >= vi0 && i <= vi1 && k >= vk0 && k <= vk1;
      e0[r] = ba[r] = bb[r] = bc[r] = bd[r] = T(0);
      if (v) {
        e0[r] = f.E[c][p];
        if (c == 0) {
          ba[r] = f.B[1][p]; bb[r] = f.B[1][p - 1];
        } else if (c == 2) {
          ba[r] = f.B[1][p]; bb[r] = f.B[1][p - g.ld];
        } else {
          ba[r] = f.B[0][p]; bb[r] = f.B[0][p - 1]; bc[r] = f.B[2][p]; bd[r] = f.B[2][p - g.ld];
        }
      }
    }
    if (!block_wait(&bar[c & 1], (c >> 1) & 1)) {
      tile_timeout(ctrl, &bar[0], &bar[1]);
      return;
    }
    if (c == 2 && ion_x != nullptr) {
      // rigid ion-column current added to Jz before the filter (each thread
      // converts its columns' factors once)
      T cz[(256 + FT_Z - 1) / FT_Z];
#pragma unroll
      for (int u = 0; u < (256 + FT_Z - 1) / FT_Z; u++) {
        const int lk = threadIdx.x + u * FT_Z, gk = gk0 + lk;
        cz[u] = (lk < tm.BZ && gk >= 0 && gk <= g.nz) ? T(ion_c[gk]) : T(0);
      }
      for (int li = threadIdx.y; li < tm.BX; li += FT_TY) {
        const int gi = gi0 + li;
        if (gi < 0 || gi > g.nx) continue;
        const T ix = T(ion_coef * ion_x[gi]);
#pragma unroll
        for (int u = 0; u < (256 + FT_Z - 1) / FT_Z; u++) {
          const int lk = threadIdx.x + u * FT_Z;
          if (lk < tm.BZ) A[li * tm.BZ + lk] += ix * cz[u];
        }
      }
      __syncthreads();
    }
    if (FILT) filter_tile<T, PT>(A + (tm.H - H) * tm.BZ + (tm.HZ - H), tm.BZ, B1, Zb, ft);
    // block-uniform: the tiles clear of the PML run the rows without its branches (no FP64 table reads)
    const bool clear = i0 >= pt.iin0 && i0 + FT_X - 1 <= pt.iin1 && k0 >= pt.kin0 && k0 + FT_Z - 1 <= pt.kin1;
    auto rows = [&](auto pml) {
      constexpr bool interior = !decltype(pml)::value;
#pragma unroll
    for (int r = 0; r < NR; r++) {
      const int ti = threadIdx.y + r * FT_TY;
      const int i = i0 + ti;
      if (i > g.nx || k > g.nz) continue;
      const long p = (long)i * g.ld + k;
      f.Jn[c][p] = T(0);
      const bool v = i >= vi0 && i <= vi1 && k >= vk0 && k <= vk1;
      if (!v) {
        f.Eo[c][p] = T(0);
        continue;
      }
      const T jv = FILT ? Zb[ti * FT_Z + threadIdx.x] : A[(ti + tm.H) * tm.BZ + threadIdx.x + tm.HZ];
      const T eo = e0[r];
      T en;
      if (c == 0) {
        T d = (ba[r] - bb[r]) * idz;
        if (!interior && pt.sz_i[k] > 0.0) en = T(pt.xz_i[k] * (double)eo - c2d * pt.cz_i[k] * (double)d);
        else en = eo - dt * (c2 * d + jv * ie0);
      } else if (c == 2) {
        T d = (ba[r] - bb[r]) * idx;
        if (!interior && pt.sx_i[i] > 0.0) en = T(pt.xx_i[i] * (double)eo + c2d * pt.cx_i[i] * (double)d);
        else en = eo + dt * (c2 * d - jv * ie0);
      } else {
        T dbx = (ba[r] - bb[r]) * idz;
        T dbz = (bc[r] - bd[r]) * idx;
        if (!interior && (pt.sx_i[i] > 0.0 || pt.sz_i[k] > 0.0)) {
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
    };
    if (clear) rows(std::false_type{});
    else rows(std::true_type{});
    __syncthreads();
  }
}

template <class T, bool FILT, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY, sizeof(T) == 4 ? 4 : 2) k_ampere(GridP g, FieldPtrs<T> f, PmlTabs pt, FilterTaps<T> ft,
                                                        const double* ion_x, const double* ion_c, double ion_coef,
                                                        const __grid_constant__ CUtensorMap mapJ, TileMaps tm,
                                                        Ctrl* ctrl) {
  ampere_tile<T, FILT, PT>(g, f, pt, ft, ion_x, ion_c, ion_coef, &mapJ, tm, ctrl, blockIdx.x, blockIdx.y);
}

// ---------------------------------------------------------------------------
// batched field kernels of an ensemble step: one block per tile of every run (tile_off: prefix sums)
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* m) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(m) : "memory");
}

template <class T, bool FRIED, bool CK>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_faraday_batch(const StepArgs<T>* a, const int* off, int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0 && threadIdx.y == 0) s_r = batch_run(off, nruns, blockIdx.x);
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  const int lb = blockIdx.x - off[s_r];
  faraday_tile<T, FRIED, CK>(A.g, A.f, A.pt, A.far, lb % A.tiles_k, lb / A.tiles_k);
}

// the fused Faraday + E filter over every run's tiles (the run's descriptors in device memory)
template <class T, bool FRIED, bool CK, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY, 4) k_faraday_fused_batch(const StepArgs<T>* a, const int* off,
                                                                     int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    s_r = batch_run(off, nruns, blockIdx.x);
    const StepArgs<T>& A0 = a[s_r];
    tensormap_acquire(&A0.tm.E[A0.mapE]);
    if (FRIED) {
      tensormap_acquire(&A0.tm.Er[1 - A0.mapE]);
      tensormap_acquire(&A0.tm.Eb[A0.mapEb]);
    }
  }
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  const int lb = blockIdx.x - off[s_r];
  faraday_fused_tile<T, FRIED, CK, PT>(A.g, A.f, A.pt, A.far, A.ft, &A.tm.E[A.mapE], &A.tm.Er[1 - A.mapE],
                                       &A.tm.Eb[A.mapEb], A.ctrl, lb % A.tiles_k, lb / A.tiles_k);
}

template <class T, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY) k_filter_fields_batch(const StepArgs<T>* a, const int* off,
                                                                     int nruns, int c_first) {
  __shared__ int s_r;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    s_r = batch_run(off, nruns, blockIdx.x);
    tensormap_acquire(&a[s_r].tm.E[a[s_r].mapE]);
    tensormap_acquire(&a[s_r].tm.Bavg);
  }
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  const int lb = blockIdx.x - off[s_r];
  filter_fields_tile<T, PT>(A.g, A.f, A.ft, &A.tm.E[A.mapE], &A.tm.Bavg, A.tm, A.ctrl, lb % A.tiles_k,
                            lb / A.tiles_k, c_first);
}

template <class T, bool FILT, int PT>
__global__ void __launch_bounds__(FT_Z* FT_TY, sizeof(T) == 4 ? 4 : 2) k_ampere_batch(const StepArgs<T>* a, const int* off, int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    s_r = batch_run(off, nruns, blockIdx.x);
    tensormap_acquire(&a[s_r].tm.J[a[s_r].mapJ]);
  }
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  const int lb = blockIdx.x - off[s_r];
  ampere_tile<T, FILT, PT>(A.g, A.f, A.pt, A.ft, A.ion_on ? A.ion_x : nullptr, A.ion_C, A.ion_coef,
                           &A.tm.J[A.mapJ], A.tm, A.ctrl, lb % A.tiles_k, lb / A.tiles_k);
}

}  // namespace

template <class T>
void launch_faraday_filter_batch(const StepArgs<T>* a, const BatchGrid& bg, bool friedman, bool ck, int pt_taps,
                                 bool filt_gather, size_t filt_smem, size_t fused_smem, cudaStream_t s) {
  dim3 blk(FT_Z, FT_TY);
  if (fused_smem > 0 && filt_gather && (pt_taps == 1 || pt_taps == 5)) {
#define FUSEDB(FR, C, PTV)                                                                                    \
  cudaFuncSetAttribute(k_faraday_fused_batch<T, FR, C, PTV>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                       (int)fused_smem);                                                                      \
  k_faraday_fused_batch<T, FR, C, PTV><<<bg.tiles, blk, fused_smem, s>>>(a, bg.tile_off, bg.nruns);
    if (pt_taps == 5) {
      if (friedman) { if (ck) { FUSEDB(true, true, 5) } else { FUSEDB(true, false, 5) } }
      else { if (ck) { FUSEDB(false, true, 5) } else { FUSEDB(false, false, 5) } }
    } else {
      if (friedman) { if (ck) { FUSEDB(true, true, 1) } else { FUSEDB(true, false, 1) } }
      else { if (ck) { FUSEDB(false, true, 1) } else { FUSEDB(false, false, 1) } }
    }
#undef FUSEDB
    // B_avg's gather copies
    if (pt_taps == 5) {
      cudaFuncSetAttribute(k_filter_fields_batch<T, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_smem);
      k_filter_fields_batch<T, 5><<<bg.tiles, blk, filt_smem, s>>>(a, bg.tile_off, bg.nruns, 3);
    } else {
      cudaFuncSetAttribute(k_filter_fields_batch<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_smem);
      k_filter_fields_batch<T, 1><<<bg.tiles, blk, filt_smem, s>>>(a, bg.tile_off, bg.nruns, 3);
    }
    return;
  }
  if (friedman) {
    if (ck) k_faraday_batch<T, true, true><<<bg.tiles, blk, 0, s>>>(a, bg.tile_off, bg.nruns);
    else k_faraday_batch<T, true, false><<<bg.tiles, blk, 0, s>>>(a, bg.tile_off, bg.nruns);
  } else {
    if (ck) k_faraday_batch<T, false, true><<<bg.tiles, blk, 0, s>>>(a, bg.tile_off, bg.nruns);
    else k_faraday_batch<T, false, false><<<bg.tiles, blk, 0, s>>>(a, bg.tile_off, bg.nruns);
  }
  if (!filt_gather) return;
#define FBATCH(PTV)                                                                                      \
  cudaFuncSetAttribute(k_filter_fields_batch<T, PTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)filt_smem); \
  k_filter_fields_batch<T, PTV><<<bg.tiles, blk, filt_smem, s>>>(a, bg.tile_off, bg.nruns, 0);
  switch (pt_taps) {
    case 1: { FBATCH(1) break; }
    case 2: { FBATCH(2) break; }
    case 3: { FBATCH(3) break; }
    case 4: { FBATCH(4) break; }
    case 5: { FBATCH(5) break; }
    case 6: { FBATCH(6) break; }
    default: { FBATCH(0) break; }
  }
#undef FBATCH
}

template <class T>
void launch_ampere_batch(const StepArgs<T>* a, const BatchGrid& bg, bool filt_J, int pt_taps, size_t amp_smem,
                         cudaStream_t s) {
  dim3 blk(FT_Z, FT_TY);
#define ABATCH(F, PTV)                                                                                   \
  cudaFuncSetAttribute(k_ampere_batch<T, F, PTV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)amp_smem); \
  k_ampere_batch<T, F, PTV><<<bg.tiles, blk, amp_smem, s>>>(a, bg.tile_off, bg.nruns);
  if (!filt_J) {
    ABATCH(false, 0)
    return;
  }
  switch (pt_taps) {
    case 1: { ABATCH(true, 1) break; }
    case 2: { ABATCH(true, 2) break; }
    case 3: { ABATCH(true, 3) break; }
    case 4: { ABATCH(true, 4) break; }
    case 5: { ABATCH(true, 5) break; }
    case 6: { ABATCH(true, 6) break; }
    default: { ABATCH(true, 0) break; }
  }
#undef ABATCH
}

void field_tiles(const GridP& g, int& tiles_k, int& tiles_i) {
  tiles_k = (g.nz + 1 + FT_Z - 1) / FT_Z;
  tiles_i = (g.nx + 1 + FT_X - 1) / FT_X;
}

template <class T>
FarK<T> faraday_coefs(double a2, double b2, double theta) {
  FarK<T> q;
  q.a2 = T(a2); q.b2 = T(b2);
  q.c1 = T(1.0 + theta / 4.0); q.c2 = T(-0.5); q.c3 = T(0.5 - theta / 4.0);
  q.h1 = T(1.0 - theta / 2.0); q.h2 = T(theta / 2.0);
  return q;
}

template <class T>
void launch_faraday(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, double a2, double b2, double theta,
                    bool friedman, cudaStream_t s) {
  const FarK<T> q = faraday_coefs<T>(a2, b2, theta);
  dim3 blk(FT_Z, FT_TY), grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X);
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
  return (2 * (size_t)tile_stride<T>(tm) + (size_t)FT_X * filter_wzp(H) + (size_t)FT_X * FT_Z) * sizeof(T) + 128;
}

template <class T>
static FilterTaps<T> make_taps(const FilterSpec& fs) {
  // compose n bilinear passes (alpha = 1/2) and the compensation pass (alpha_c = n/2 + 1) at one stride, or,
  // for a wide-band filter, at each stride of the set in turn, into one tap array
  const int P = fs.passes + (fs.compensate ? 1 : 0);
  FilterTaps<T> ft;
  if (fs.strides[0] <= 0) {
    double k[2 * FILTER_HMAX + 1] = {0.0};
    int len = 1;
    k[0] = 1.0;
    for (int p = 0; p < P; p++) {
      const double al = p < fs.passes ? 0.5 : 0.5 * fs.passes + 1.0;
      const double be = 0.5 * (1.0 - al);
      double r[2 * FILTER_HMAX + 1] = {0.0};
      for (int j = 0; j < len; j++) {
        r[j] += be * k[j];
        r[j + 1] += al * k[j];
        r[j + 2] += be * k[j];
      }
      len += 2;
      for (int j = 0; j < len; j++) k[j] = r[j];
    }
    ft.P = P;
    ft.s = fs.stride;
    ft.H = P * fs.stride;
    for (int j = 0; j < 2 * FILTER_HMAX + 1; j++) ft.c[j] = T(j < len ? k[j] : 0.0);
    return ft;
  }
  const int H = filter_halo(fs);
  double k[2 * FILTER_HMAX + 1] = {0.0};   // offsets -H..H
  k[H] = 1.0;
  for (int q = 0; q < 4 && fs.strides[q] > 0; q++) {
    const int st = fs.strides[q];
    for (int p = 0; p < P; p++) {
      const double al = p < fs.passes ? 0.5 : 0.5 * fs.passes + 1.0;
      const double be = 0.5 * (1.0 - al);
      double r[2 * FILTER_HMAX + 1] = {0.0};
      for (int j = 0; j <= 2 * H; j++) {
        if (k[j] == 0.0) continue;
        r[j] += al * k[j];
        if (j - st >= 0) r[j - st] += be * k[j];
        if (j + st <= 2 * H) r[j + st] += be * k[j];
      }
      for (int j = 0; j <= 2 * H; j++) k[j] = r[j];
    }
  }
  ft.P = H;
  ft.s = 1;
  ft.H = H;
  for (int j = 0; j < 2 * FILTER_HMAX + 1; j++) ft.c[j] = T(j <= 2 * H ? k[j] : 0.0);
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

// 3D tensor over a 3-component block: (nz+1) x (nx+1) x 3, rows ld elements apart, components cs apart;
// boxes of bx rows by bz columns (the tile maps' BX x BZ by default)
template <class T>
static bool encode_block(CUtensorMap* m, const void* base, const GridP& g, const TileMaps& tm, int bx = 0,
                         int bz = 0) {
  EncodeTiledFn fn = encode_fn();
  if (!fn || !base) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)(g.nz + 1), (cuuint64_t)(g.nx + 1), 3};
  const cuuint64_t strides[2] = {(cuuint64_t)g.ld * sizeof(T), (cuuint64_t)g.cs * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)(bz ? bz : tm.BZ), (cuuint32_t)(bx ? bx : tm.BX), 1};
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
  tm.ok = tm.r_ok = false;
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
  // the fused Faraday kernel's small boxes of E^{n-1} and of Friedman's E-bar (FT_X + 2 by FT_Z + 8)
  tm.Ebbase[0] = f.Eb[0];
  tm.Ebbase[1] = f.Ebn[0];
  tm.r_ok = f.Eb[0] && f.Ebn[0] && encode_block<T>(&tm.Er[0], f.E[0], g, tm, FT_X + 2, FT_Z + 8) &&
            encode_block<T>(&tm.Er[1], f.Eo[0], g, tm, FT_X + 2, FT_Z + 8) &&
            encode_block<T>(&tm.Eb[0], f.Eb[0], g, tm, FT_X + 2, FT_Z + 8) &&
            encode_block<T>(&tm.Eb[1], f.Ebn[0], g, tm, FT_X + 2, FT_Z + 8);
  return ok;
}

// compile-time tap count for the common stride-1 filters; 0 = runtime loops
template <class T>
static int filter_pt(const FilterTaps<T>& ft) { return (ft.s == 1 && ft.P >= 1 && ft.P <= 6) ? ft.P : 0; }

template <class T, int PT>
static void run_filter_fields(dim3 grd, dim3 blk, size_t sm, cudaStream_t s, const GridP& g, const FieldPtrs<T>& f,
                              const FilterTaps<T>& ft, const CUtensorMap& mE, const TileMaps& tm, Ctrl* ctrl,
                              int c_first) {
  cudaFuncSetAttribute(k_filter_fields<T, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_filter_fields<T, PT><<<grd, blk, sm, s>>>(g, f, ft, mE, tm.Bavg, tm, ctrl, c_first);
}

template <class T>
void launch_filter_fields(const GridP& g, const FieldPtrs<T>& f, const FilterSpec& fs, bool enabled,
                          const TileMaps& tm, Ctrl* ctrl, cudaStream_t s, int c_first) {
  if (!enabled) return;
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  const size_t sm = tile_smem<T>(tm, ft.H);
  const CUtensorMap& mE = tm.Ebase[0] == (const void*)f.E[0] ? tm.E[0] : tm.E[1];
  switch (filter_pt(ft)) {
    case 1: run_filter_fields<T, 1>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    case 2: run_filter_fields<T, 2>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    case 3: run_filter_fields<T, 3>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    case 4: run_filter_fields<T, 4>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    case 5: run_filter_fields<T, 5>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    case 6: run_filter_fields<T, 6>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
    default: run_filter_fields<T, 0>(grd, blk, sm, s, g, f, ft, mE, tm, ctrl, c_first); break;
  }
}

// shared memory of the fused Faraday kernel: four staged boxes, E_eff, the filter's scratch
template <class T>
static size_t fused_smem(const TileMaps& tm, int H, bool fried) {
  // three E^n boxes, then the E^{n-1}/E-bar boxes, whose space the filter's scratch reuses
  const size_t scratch = (size_t)FT_X * filter_wzp(H) + (size_t)FT_X * FT_Z;
  const size_t rest = fried ? std::max(6 * (size_t)ring_stride<T>(), scratch) : scratch;
  return (3 * (size_t)tile_stride<T>(tm) + rest) * sizeof(T) + 128;
}

template <class T>
size_t faraday_fused_smem(const TileMaps& tm, int H, int pt_taps, bool friedman) {
  if (!tm.ok || (friedman && !tm.r_ok) || H != tm.H || (pt_taps != 1 && pt_taps != 5)) return 0;
  const size_t sm = fused_smem<T>(tm, H, friedman);
  return sm <= 227 * 1024 ? sm : 0;
}

template <class T, bool FRIED, bool CK, int PT>
static bool run_faraday_fused(dim3 grd, dim3 blk, cudaStream_t s, const GridP& g, const FieldPtrs<T>& f,
                              const PmlTabs& pt, const FarK<T>& q, const FilterTaps<T>& ft, const TileMaps& tm,
                              Ctrl* ctrl) {
  const size_t sm = fused_smem<T>(tm, ft.H, FRIED);
  if (sm > 227 * 1024) return false;
  const bool cur0 = tm.Ebase[0] == (const void*)f.E[0];
  const CUtensorMap& mE = cur0 ? tm.E[0] : tm.E[1];
  const CUtensorMap& mEo = cur0 ? tm.Er[1] : tm.Er[0];
  const CUtensorMap& mEb = tm.Ebbase[0] == (const void*)f.Eb[0] ? tm.Eb[0] : tm.Eb[1];
  cudaFuncSetAttribute(k_faraday_fused<T, FRIED, CK, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_faraday_fused<T, FRIED, CK, PT><<<grd, blk, sm, s>>>(g, f, pt, q, ft, mE, mEo, mEb, ctrl);
  return true;
}

// Faraday fused with the gather filter of E (TMA-staged E tiles). False when the fused kernel does not
// apply (no gather filter, a strided filter, other than one or five passes, E-bar descriptors missing):
// the caller then runs launch_faraday and launch_filter_fields over all six components.
template <class T>
bool launch_faraday_fused(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, double a2, double b2,
                          double theta, bool friedman, const FilterSpec& fs, bool filt_gather, const TileMaps& tm,
                          Ctrl* ctrl, cudaStream_t s) {
  if (!filt_gather || !tm.ok || (friedman && !tm.r_ok)) return false;
  const FilterTaps<T> ft = make_taps<T>(fs);
  const int ptc = filter_pt(ft);
  if (ft.H != tm.H) return false;
  const FarK<T> q = faraday_coefs<T>(a2, b2, theta);
  dim3 blk(FT_Z, FT_TY), grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X);
  const bool ck = b2 != 0.0;
  // one pass (the single binomial pass) and five (four passes and the compensation)
  if (ptc == 5) {
    if (friedman) {
      if (ck) return run_faraday_fused<T, true, true, 5>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
      return run_faraday_fused<T, true, false, 5>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
    }
    if (ck) return run_faraday_fused<T, false, true, 5>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
    return run_faraday_fused<T, false, false, 5>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
  }
  if (ptc == 1) {
    if (friedman) {
      if (ck) return run_faraday_fused<T, true, true, 1>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
      return run_faraday_fused<T, true, false, 1>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
    }
    if (ck) return run_faraday_fused<T, false, true, 1>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
    return run_faraday_fused<T, false, false, 1>(grd, blk, s, g, f, pt, q, ft, tm, ctrl);
  }
  return false;
}

template <class T, bool FILT, int PT>
static void run_ampere(dim3 grd, dim3 blk, size_t sm, cudaStream_t s, const GridP& g, const FieldPtrs<T>& f,
                       const PmlTabs& pt, const FilterTaps<T>& ft, const double* ion_x, const double* ion_c,
                       double ion_coef, const CUtensorMap& mJ, const TileMaps& tm, Ctrl* ctrl) {
  cudaFuncSetAttribute(k_ampere<T, FILT, PT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_ampere<T, FILT, PT><<<grd, blk, sm, s>>>(g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl);
}

template <class T>
void launch_ampere(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, const FilterSpec& fs, bool filter_on,
                   const double* ion_x, const double* ion_c, double ion_coef, const TileMaps& tm, Ctrl* ctrl,
                   cudaStream_t s) {
  const FilterTaps<T> ft = make_taps<T>(fs);
  dim3 grd((g.nz + 1 + FT_Z - 1) / FT_Z, (g.nx + 1 + FT_X - 1) / FT_X), blk(FT_Z, FT_TY);
  const CUtensorMap& mJ = tm.Jbase[0] == (const void*)f.J[0] ? tm.J[0] : tm.J[1];
  const size_t sm = tile_smem<T>(tm, filter_on ? ft.H : 0);
  if (!filter_on) {
    run_ampere<T, false, 0>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl);
    return;
  }
  switch (filter_pt(ft)) {
    case 1: run_ampere<T, true, 1>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    case 2: run_ampere<T, true, 2>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    case 3: run_ampere<T, true, 3>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    case 4: run_ampere<T, true, 4>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    case 5: run_ampere<T, true, 5>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    case 6: run_ampere<T, true, 6>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
    default: run_ampere<T, true, 0>(grd, blk, sm, s, g, f, pt, ft, ion_x, ion_c, ion_coef, mJ, tm, ctrl); break;
  }
}

template void launch_faraday<float>(const GridP&, const FieldPtrs<float>&, const PmlTabs&, double, double, double,
                                    bool, cudaStream_t);
template void launch_faraday<double>(const GridP&, const FieldPtrs<double>&, const PmlTabs&, double, double, double,
                                     bool, cudaStream_t);
template <class T>
FilterTaps<T> filter_taps(const FilterSpec& fs) { return make_taps<T>(fs); }
template <class T>
int filter_taps_class(const FilterTaps<T>& ft) { return filter_pt<T>(ft); }
template <class T>
size_t tile_smem_bytes(const TileMaps& tm, int H) { return tile_smem<T>(tm, H); }

#define INSTF(T)                                                                                                 \
  template FarK<T> faraday_coefs<T>(double, double, double);                                                     \
  template FilterTaps<T> filter_taps<T>(const FilterSpec&);                                                      \
  template int filter_taps_class<T>(const FilterTaps<T>&);                                                       \
  template size_t tile_smem_bytes<T>(const TileMaps&, int);                                                      \
  template void launch_faraday_filter_batch<T>(const StepArgs<T>*, const BatchGrid&, bool, bool, int, bool, size_t, \
                                               size_t, cudaStream_t);                                           \
  template void launch_ampere_batch<T>(const StepArgs<T>*, const BatchGrid&, bool, int, size_t, cudaStream_t);      \
  template bool make_tile_maps<T>(const GridP&, const FieldPtrs<T>&, int, TileMaps&);                            \
  template void launch_filter_fields<T>(const GridP&, const FieldPtrs<T>&, const FilterSpec&, bool, const TileMaps&, \
                                        Ctrl*, cudaStream_t, int);                                               \
  template size_t faraday_fused_smem<T>(const TileMaps&, int, int, bool);                                          \
  template bool launch_faraday_fused<T>(const GridP&, const FieldPtrs<T>&, const PmlTabs&, double, double, double,  \
                                        bool, const FilterSpec&, bool, const TileMaps&, Ctrl*, cudaStream_t);   \
  template void launch_ampere<T>(const GridP&, const FieldPtrs<T>&, const PmlTabs&, const FilterSpec&, bool,       \
                                 const double*, const double*, double, const TileMaps&, Ctrl*, cudaStream_t);
INSTF(float)
INSTF(double)
#undef INSTF

}  // namespace picgb
