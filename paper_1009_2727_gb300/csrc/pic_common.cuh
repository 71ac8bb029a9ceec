// Internal declarations of the GB300 PIC library (device types, shape
// functions, kernel launchers). Not part of the public ABI (include/pic.h).
#pragma once

#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

namespace picgb {

// CODATA 2018
constexpr double kC = 299792458.0;
constexpr double kQe = 1.602176634e-19;
constexpr double kMe = 9.1093837015e-31;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kPi = 3.14159265358979323846;

enum Comp { EX = 0, EY, EZ, BX, BY, BZ };

// Device status bits (sticky, read by pic_sync)
enum StatusBits : int { ST_OVERFLOW = 1, ST_NAN = 2, ST_OUTSIDE = 4, ST_TIMEOUT = 8 };

// Geometry passed by value to every kernel.
struct GridP {
  int nx, nz, ld;            // cells; row stride (elements) of every grid array
  long cs;                   // stride between the components of a 3-component block
  double dx, dz, dt;
  double idx, idz;           // 1/dx, 1/dz from the host
  float dtf, idxf, idzf;     // dt, 1/dx, 1/dz in FP32 (the field kernels of the mixed path run no FP64)
  double z0;                 // grid origin along z (moving window)
  int gx_lo, gx_hi, gz_lo, gz_hi;  // particle domain (cells)
  int pml;                   // PML cells (0 = none)
  // mixed path: particle z is stored in the frame drifting with the plasma
  // (-beta c); grid z = stored z - S with S = beta c t / dz = fr_sz + fr_fz
  // (fr_sz modulo 2^16, fr_fz in [0, 1)) at the time of the stored positions
  int fr_sz;
  float fr_fz;
  // mixed path: u_z is stored as u_z - fr_u0, fr_u0 = -gamma beta c (FP32), the
  // plasma drift momentum, so that its changes keep FP32 precision
  float fr_u0;
  // mixed path: the plasma lattice (rows of il_nxl particles, il_ppcx x il_ppcz
  // per cell); the stored particle id is (row << il_kb) | column; the grid
  // origin in cells (moving window shifts)
  int il_nxl, il_ppcx, il_ppcz, il_kb;
  int z0_cells;
};

// dt, 1/dx, 1/dz in the path's type (host-computed: on this GPU an FP64 divide or conversion per thread
// would run on its narrow FP64 pipe)
template <class T>
__host__ __device__ __forceinline__ T grid_dt(const GridP& g) {
  if constexpr (sizeof(T) == 4) return g.dtf; else return g.dt;
}
template <class T>
__host__ __device__ __forceinline__ T grid_idx(const GridP& g) {
  if constexpr (sizeof(T) == 4) return g.idxf; else return g.idx;
}
template <class T>
__host__ __device__ __forceinline__ T grid_idz(const GridP& g) {
  if constexpr (sizeof(T) == 4) return g.idzf; else return g.idz;
}

// Valid index range of each E/B component (PEC walls); J uses the E ranges.
__host__ __device__ inline void valid_range(int comp, int nx, int nz, int& i0, int& i1, int& k0, int& k1) {
  switch (comp) {
    case EX: i0 = 0; i1 = nx - 1; k0 = 1; k1 = nz - 1; break;
    case EY: i0 = 1; i1 = nx - 1; k0 = 1; k1 = nz - 1; break;
    case EZ: i0 = 1; i1 = nx - 1; k0 = 0; k1 = nz - 1; break;
    case BX: i0 = 0; i1 = nx;     k0 = 0; k1 = nz - 1; break;
    case BY: i0 = 0; i1 = nx - 1; k0 = 0; k1 = nz - 1; break;
    default: i0 = 0; i1 = nx - 1; k0 = 0; k1 = nz;     break;
  }
}

// PML coefficient tables (always FP64): sigma, xi and (1-xi)/sigma at integer
// and half positions along x (size nx+1) and z (size nz+1).
struct PmlTabs {
  const double *sx_i, *sx_h, *xx_i, *xx_h, *cx_i, *cx_h;
  const double *sz_i, *sz_h, *xz_i, *xz_h, *cz_i, *cz_h;
  int iin0, iin1, kin0, kin1;   // nodes whose sigma is zero at both staggerings (the interior)
};

template <class T>
struct FieldPtrs {
  T* E[3];      // E^n
  T* Eo[3];     // other E buffer: E^{n-1} on entry to Faraday, receives E^{n+1} in Ampere
  T* B[3];
  T* J[3];      // current being deposited this step
  T* Jn[3];     // other current buffer (zeroed by Ampere for the next step)
  T* Eb[3];     // Friedman E-bar (read)
  T* Ebn[3];    // Friedman E-bar (write)
  T* Bavg[3];   // (B^{n-1/2} + B^{n+1/2})/2
  T* fE[3];     // gather copies
  T* fB[3];
  T* nE[3];     // 'momentum conserving' gather: the copies interpolated to the nodes (3 x cs each, contiguous)
  T* nB[3];
  T* Byx; T* Byz; T* Eyx; T* Eyz;  // split PML parts (full-size, used in the PML only)
};

struct FilterSpec {
  int passes, stride, compensate;
  int strides[4];   // wide-band filter: the passes repeated at each of these strides (0-terminated); else none
};

// total halo of the filter along one axis: (passes + compensation) times the sum of its strides
inline int filter_halo(const FilterSpec& fs) {
  const int P = fs.passes + (fs.compensate ? 1 : 0);
  int ss = fs.stride;
  if (fs.strides[0] > 0) {
    ss = 0;
    for (int q = 0; q < 4 && fs.strides[q] > 0; q++) ss += fs.strides[q];
  }
  return P * ss;
}
constexpr int FILTER_HMAX = 40;

// composed taps of the multi-pass filter along one axis: c[j] at offset (j - P) * s, j = 0..2P (a wide-band
// filter is stored densely: s = 1, P = H)
template <class T>
struct FilterTaps {
  T c[2 * FILTER_HMAX + 1];
  int P, s, H;
};

// Particle chunk: a contiguous particle range and the bounding box of the
// cells its particles occupy (inclusive, grid-relative cells).
struct Chunk {
  int p0, p1;
  int ix0, ix1, iz0, iz1;
};

// Particle storage (structure of arrays). The FP64 path keeps absolute
// positions; the mixed path keeps a cell (iz | ix << 16) and the FP32 offset
// inside it, so that its push needs no FP64 arithmetic. Its z is kept in the
// frame drifting with the plasma (see GridP::fr_sz): a particle at the plasma
// drift never changes its stored z, so the cold plasma keeps its place against
// the rigid ions exactly instead of accumulating FP32 rounding every step.
template <class T>
struct Particles {
  double* x; double* z;          // FP64 path [m]
  uint32_t* cell;                // mixed path
  float* ox; float* oz;          // mixed path, offsets in [0, 1)
  T* ux; T* uy; T* uz; T* w;
  uint32_t* id;
};
template <class T>
struct CellPos { static constexpr bool value = false; };
template <>
struct CellPos<float> { static constexpr bool value = true; };

__host__ __device__ inline uint32_t pack_cell(int ix, int iz) { return (uint32_t)iz | ((uint32_t)ix << 16); }
__host__ __device__ inline int cell_x(uint32_t c) { return (int)(c >> 16); }
__host__ __device__ inline int cell_z(uint32_t c) { return (int)(c & 0xffffu); }

// mixed path: grid cell and in-cell offset along z of a particle stored in the
// drifting frame, for the frame shift (sz, fz) (the stored cell is taken
// modulo 2^16, so S may grow without bound)
__host__ __device__ inline void frame_z(uint32_t c, float oz, int sz, float fz, int& iz, float& tz) {
  float t = oz - fz;
  int b = 0;
  if (t < 0.0f) {
    t += 1.0f;
    b = 1;
    if (t >= 1.0f) { t = 0.0f; b = 0; }
  }
  iz = (cell_z(c) - sz - b) & 0xffff;
  tz = t;
}

// Lattice site (row m, column a) of a plasma particle: the stored cell and
// offsets (z in the drifting frame) that the particle gets at injection, and
// that its lab-fixed ion keeps for ever (row m at z = (m + 1/2) dz / ppcz).
// Integer arithmetic and FP32 divisions of small integers: for power-of-two
// ppcx, ppcz these are exact, so lattice_site_pow2 (shifts) gives the same bits.
__host__ __device__ inline void lattice_site(int m, int a, int ppcx, int ppcz, int gx_lo, int z0_cells,
                                             uint32_t& cell, float& ox, float& oz) {
  const int n2 = 2 * m + 1, d2 = 2 * ppcz;
  cell = pack_cell(gx_lo + a / ppcx, (n2 / d2 - z0_cells) & 0xffff);
  oz = (float)(n2 % d2) / (float)d2;
  ox = ((float)(a % ppcx) + 0.5f) / (float)ppcx;
}
// the same for ppcx = 2^lpx, ppcz = 2^lpz, from the stored id (row << kb) | column
__host__ __device__ inline void lattice_site_pow2(uint32_t id, int kb, int lpx, int lpz, int gx_lo, int z0_cells,
                                                  uint32_t& cell, float& ox, float& oz) {
  const int m = (int)(id >> kb), a = (int)(id & ((1u << kb) - 1u));
  const int n2 = 2 * m + 1;
  cell = pack_cell(gx_lo + (a >> lpx), ((n2 >> (lpz + 1)) - z0_cells) & 0xffff);
  oz = (float)(n2 & ((2 << lpz) - 1)) * (1.0f / (float)(2 << lpz));
  ox = ((float)(a & ((1 << lpx) - 1)) + 0.5f) * (1.0f / (float)(1 << lpx));
}

// frame shift S (cells, FP64) -> (S mod 2^16 integer part, FP32 fraction)
inline void frame_of(double S, int& sz, float& fz) {
  const double fl = __builtin_floor(S);
  float f = (float)(S - fl);
  long long si = (long long)fl;
  if (f >= 1.0f) { f = 0.0f; si += 1; }
  sz = (int)(si & 0xffff);
  fz = f;
}

// Control block in device memory.
struct Ctrl {
  int count;          // particle slots in use (electrons)
  int nchunks;
  int next_chunk;     // work counter of the persistent particle kernel
  int status;
  int overflow_chunks;
  int n_defer;        // particles of this step's push left for the global-memory pass
  int n_ovf;          // chunks of this step's push left for the global-memory pass (window too large)
  int pad;
  double red[8];      // reduction scratch
};

// Constants of the particle push (one run, one step).
struct PushConst {
  double dx, dz, dt, z0;            // FP64 path
  double xlo, xhi, zlo, zhi;        // FP64 path removal bounds [m]
  int cx_lo, cx_hi, cz_lo, cz_hi;   // mixed path removal bounds [cells, hi exclusive]
  float dtdx, dtdz;                 // mixed path
  double qm_half;                   // q dt/(2m)
  double kx, kz, ky;                // deposit: -q/(dz dt), -q/(dx dt), q/(dx dz)
  float qm_half_f, kx_f, kz_f, ky_f;  // the same in FP32 for the mixed path
  // mixed path: the plasma drift momentum u0 = -gamma beta c (FP32) and gamma0; the
  // frame shift (GridP::fr_sz) at t^n and t^{n+1}
  float u0z_f, g0_f, g0sq_f;
  int fr0_sz, fr1_sz;
  float fr0_fz, fr1_fz;
  // mixed path with lab-fixed ions: each electron carries the ion of its lattice
  // site (pairs; power-of-two particles per cell); ion rows below mlo have left
  // the particle domain; the stored id is (row << kb) | column
  int pairs, mlo;
  int kb, lpx, lpz, gx_lo, z0_cells;
};

// Coefficients of the Faraday update (Eq. Faraday_Friedman, reduced to 2D).
template <class T>
struct FarK {
  T a2, b2;          // 2D reduced coefficients: alpha + 2 beta, beta + 2 gamma
  T c1, c2, c3;      // E_eff = c1 E^n + c2 E^{n-1} + c3 E-bar
  T h1, h2;          // E-bar' = h1 E^n + h2 E-bar
};

// ---------------------------------------------------------------------------
// B-spline weights from the fractional offset t in [0,1) of a position above
// node f: order 3 -> nodes f-1..f+2, order 1 -> nodes f, f+1.
template <class R>
__device__ __forceinline__ void weights3(R t, R* w) {
  R t2 = t * t, t3 = t2 * t, s = R(1) - t;
  w[0] = s * s * s * R(1.0 / 6.0);
  w[1] = R(2.0 / 3.0) - t2 + R(0.5) * t3;
  w[2] = R(1.0 / 6.0) + R(0.5) * (t + t2 - t3);
  w[3] = t3 * R(1.0 / 6.0);
}
template <class R>
__device__ __forceinline__ void weights1(R t, R* w) {
  w[0] = R(1) - t;
  w[1] = t;
}

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files, instantiated for float and double).
template <class T>
void launch_faraday(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, double a2, double b2,
                    double theta, bool friedman, cudaStream_t s);
// TMA descriptors of the 3-component blocks read by the tile kernels (a 3D tensor
// (nz+1) x (nx+1) x 3 per block; out-of-range elements read as zero)
struct TileMaps {
  CUtensorMap E[2];     // the two E buffers
  CUtensorMap J[2];     // the two current buffers
  CUtensorMap Bavg;
  CUtensorMap Er[2];    // the two E buffers in small boxes (tile + one node, z aligned), when r_ok
  CUtensorMap Eb[2];    // the two Friedman E-bar buffers in the same small boxes, when r_ok
  const void* Ebase[2];
  const void* Jbase[2];
  const void* Ebbase[2];
  int H, HZ, BX, BZ;    // halo (cells), aligned z halo, box extents
  bool ok, r_ok;
};
template <class T>
bool make_tile_maps(const GridP& g, const FieldPtrs<T>& f, int H, TileMaps& tm);
// the gather filter of components c_first..5 (E^n: 0..2, B_avg: 3..5)
template <class T>
void launch_filter_fields(const GridP& g, const FieldPtrs<T>& f, const FilterSpec& fs, bool enabled,
                          const TileMaps& tm, Ctrl* ctrl, cudaStream_t s, int c_first = 0);
// Faraday fused with the gather filter of E^n (false: not applicable, nothing launched)
template <class T>
bool launch_faraday_fused(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, double a2, double b2,
                          double theta, bool friedman, const FilterSpec& fs, bool filt_gather, const TileMaps& tm,
                          Ctrl* ctrl, cudaStream_t s);
template <class T>
void launch_ampere(const GridP& g, const FieldPtrs<T>& f, const PmlTabs& pt, const FilterSpec& fs, bool filter_on,
                   const double* ion_x, const double* ion_c, double ion_coef, const TileMaps& tm, Ctrl* ctrl,
                   cudaStream_t s);

// The push runs in two launches: the shared-memory window kernel over every chunk, then a global-memory
// pass over what it left (particles outside their chunk's box, chunks whose window exceeds the shared
// memory), recorded in defer (particle, chunk) and ovf (chunk) lists of the given capacities.
struct PushDefer {
  int2* defer;
  int* ovf;
  int defer_cap, ovf_cap;
};
template <class T>
void launch_push(const GridP& g, const FieldPtrs<T>& f, Particles<T> p, Chunk* chunks, Ctrl* ctrl, int order,
                 int grid_blocks, int smem_nodes, int tile_z, double q, double m, double gamma_b, double beta_b,
                 int fr1_sz, float fr1_fz, int pairs, int mlo, int nodal, const PushDefer& pd, cudaStream_t s);

struct SortBufs {
  int* cell_cnt;       // ntiles*tx*tz, cells in tile-major order: particles per cell
  int* cell_start;     // ntiles*tx*tz: first entry of the cell in dest
  int* tile_cnt;       // ntiles + 1
  int* tile_start;     // ntiles + 1
  int* key;            // per particle: tile-major cell (-1: dropped)
  int* slot;           // per particle: rank in its cell
  int* dest;           // per (cell, rank) entry: destination index
  int* scan_tmp;
  int ntx, ntz, tx, tz, R;
};
template <class T>
void launch_sort(const GridP& g, Particles<T> src, Particles<T> dst, SortBufs sb, Chunk* chunks, Ctrl* ctrl,
                 int cap, int chunk_max, int chunk_cap, cudaStream_t s);

struct InjectP {
  long long m_beg, m_end;       // lattice rows to create
  double t;                     // time of the positions
  double h;                     // row spacing
  double gamma, beta;
  double n0, z_start_lab, ramp_lab, length_lab;
  int ppc_x, ppc_z, nxl;
  int xblock;                   // cells per chunk along x
  int rblock;                   // rows per chunk
};
template <class T>
void launch_inject(const GridP& g, Particles<T> p, Chunk* chunks, Ctrl* ctrl, const InjectP& ip, int cap,
                   int chunk_cap, cudaStream_t s);
void launch_add_counts(Ctrl* ctrl, int dcount, int dchunks, cudaStream_t s);

void launch_ion_column(const GridP& g, long long mlo, long long mhi, double t0, double t1, const InjectP& ip,
                       int order, double* C, cudaStream_t s);
// row densities R(k) of the rigid ions at time t (for the charge density)
void launch_ion_rows(const GridP& g, long long mlo, long long mhi, double t, const InjectP& ip, int order, double* R,
                     cudaStream_t s);

struct LaserP {
  double lambda0, a0, w0, tau, t_peak, x_center, phase, z_antenna, beta_s;
  double gamma, beta;
};
// antenna current of one step: K_y(i) = amp * xs[i] on the rows k0 .. k0+7 with weights wz (1/dz included)
struct AntennaStep {
  double amp;
  int k0;
  double wz[8];
};
template <class T>
void launch_antenna(const GridP& g, T* Jy, const double* xs, const AntennaStep& a, cudaStream_t s);

template <class T>
struct Beam {
  double* x; double* z; T* ux; T* uy; T* uz;
  double* tc; double* zf0; T* uxb; T* uyb; T* uzb; int* flag;  // bit0 alive, bit1 active
  int n;
  int self;   // 1: the beam deposits its current (frozen and active particles); weights in w
  T* w;
};
template <class T>
void launch_beam_init(Beam<T> b, const double* lx, const double* lz, const double* lux, const double* luy,
                      const double* luz, double t_lab, double z_plane, double gamma, double beta, double t_now,
                      double* scratch, cudaStream_t s);
template <class T>
void launch_beam_push(const GridP& g, const FieldPtrs<T>& f, Beam<T> b, int order, double tn, double tn1, int nodal,
                      const double* scratch, cudaStream_t s);
// the frozen beam's self-field (Sec. 3.1.1) added to E (now) and B_y (half a step earlier); acc[2] is the
// beam's mean velocity; rho, tmp: (nx+1)(nz+1) doubles of scratch; tabx, tabz: sin(pi t / N) for t < 2N
template <class T>
void launch_beam_self_field(const GridP& g, const FieldPtrs<T>& f, Beam<T> b, int order, const double* acc,
                            double gv2, double* rho, double* tmp, double* tabx, double* tabz, cudaStream_t s);
// 'momentum conserving' gather (Sec. 5): f.nE / f.nB = the gather copies interpolated to the nodes
template <class T>
void launch_nodal(const GridP& g, const FieldPtrs<T>& f, cudaStream_t s);

template <class T>
void launch_btd(const GridP& g, const FieldPtrs<T>& f, int which, int post, int r0, int r1, const int* order_idx,
                const double* tp, const double* zp, double ta, double gamma, double beta, T* out, int* done,
                cudaStream_t s);

template <class T>
void launch_rho(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int order, double q, double* rho,
                cudaStream_t s);
void launch_ion_rho(const GridP& g, const double* ion_x, const double* R, double coef, double* rho, cudaStream_t s);
template <class T>
void launch_stats(const GridP& g, const FieldPtrs<T>& f, Particles<T> p, const Ctrl* ctrl, int cap, Beam<T> b,
                  double gamma, double beta, double trap, double* out, cudaStream_t s);
template <class T>
void launch_shift(const GridP& g, T* arr, T* tmp, int sh, int comp, cudaStream_t s);
void launch_shift_chunks(Chunk* chunks, Ctrl* ctrl, int sh, int chunk_cap, cudaStream_t s);
template <class T>
void launch_convert(const T* src, double* dst, const GridP& g, cudaStream_t s);
template <class T>
void launch_convert_back(const double* src, T* dst, const GridP& g, cudaStream_t s);
template <class T>
void launch_compact_copy(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, double* out6, uint32_t* id_out,
                         int* nout, cudaStream_t s);
template <class T>
void launch_shift_particles(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int sh, cudaStream_t s);
// returns 0, or 1 (nz above the scratch size), 2 (scratch address lookup failed), 3 (launch error); *why is
// the CUDA error of cases 2 and 3, *kernels the number of kernels enqueued
template <class T>
int launch_rho_noalloc(const GridP& g, Particles<T> p, const Ctrl* ctrl, int cap, int order, bool ions,
                       long long mlo, long long mhi, double t, const InjectP& ip, const double* ion_x, double* dst,
                       cudaStream_t s, cudaError_t* why, int* kernels);

// ---------------------------------------------------------------------------
// Batched step of an ensemble: every run's arguments for one step in one block of device memory, and one
// launch per kernel class over all runs (blocks partitioned among the runs; the push pulls (run, chunk)
// pairs from one queue). The host fills the blocks from the same decisions as a single run's step.
template <class T>
struct StepArgs {
  TileMaps tm;                 // TMA descriptors (first: aligned as CUtensorMap requires)
  int mapE, mapJ, mapEb;       // which E / J / E-bar descriptor is current
  GridP g;
  FieldPtrs<T> f;
  PmlTabs pt;
  FarK<T> far;
  FilterTaps<T> ft;
  int filt_gather, filt_J;
  int tiles_k, tiles_i;        // tile grid of the field kernels
  // push
  PushConst pc;
  Particles<T> p;
  Chunk* chunks;
  Ctrl* ctrl;
  PushDefer pd;
  int push_on;
  // antenna (K_y on rows k0..k0+7)
  int ant_on;
  AntennaStep ast;
  const double* ant_xs;
  // rigid-ion column current (runs without electron-ion pairs)
  int ion_on, ion_order;
  long long ion_mlo, ion_mhi;
  double ion_t0, ion_t1, ion_coef;
  double* ion_C;
  const double* ion_x;
  // plasma rows entering through the +z plane
  int inj_on, inj_xblocks;
  InjectP ip;
  int cap, chunk_cap, add_count, add_chunks;
  // test beam (pushed after the plasma, before the antenna)
  int beam_on, beam_order;
  Beam<T> beam;
  double beam_tn, beam_tn1;
  const double* beam_acc;
};

// run of a block of a batched launch: the last r with off[r] <= b (off: nruns + 1 prefix sums)
__device__ __forceinline__ int batch_run(const int* off, int nruns, int b) {
  int lo = 0, hi = nruns - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// per-run block offsets of the batched launches (prefix sums, nruns + 1 entries each, in device memory)
struct BatchGrid {
  const int* tile_off;     // field-kernel tiles
  const int* ion_off;      // ion-column blocks
  const int* inj_off;      // injection blocks
  const int* ant_off;      // antenna blocks
  int nruns, tiles, ion_blocks, inj_blocks, ant_blocks;
  int* push_counter;       // the push's (run, chunk) queue head
};
// the push's constants for one step (q, m: charge and mass; fr1: frame shift at t^{n+1}; pairs, mlo: the
// electron-ion pairs and the first live ion row)
PushConst push_const(const GridP& g, double q, double m, double gamma_b, int fr1_sz, float fr1_fz, int pairs,
                     int mlo);
// tile grid of the field kernels (tiles along z, along x) and their Faraday coefficients
void field_tiles(const GridP& g, int& tiles_k, int& tiles_i);
template <class T>
FarK<T> faraday_coefs(double a2, double b2, double theta);
// Faraday (+ Friedman, PML) and the gather-field filter over every run's tiles
// fused_smem > 0: Faraday fused with the E filter (every run's descriptors allow it), then the filter of
// B_avg only
template <class T>
void launch_faraday_filter_batch(const StepArgs<T>* a, const BatchGrid& bg, bool friedman, bool ck, int pt_taps,
                                 bool filt_gather, size_t filt_smem, size_t fused_smem, cudaStream_t s);
// shared memory of the fused Faraday kernel for these tile maps and filter halo, 0 when it does not apply
template <class T>
size_t faraday_fused_smem(const TileMaps& tm, int H, int pt_taps, bool friedman);
// the push's window kernel over every run's chunks (one queue), then its global-memory pass
template <class T>
void launch_push_batch(const StepArgs<T>* a, const BatchGrid& bg, int order, int grid_blocks, int smem_nodes,
                       int tile_z, cudaStream_t s);
// the antenna and the rigid-ion column current of every run
template <class T>
void launch_antenna_ion_batch(const StepArgs<T>* a, const BatchGrid& bg, bool any_ion, cudaStream_t s);
// the current filter + Ampere (+ PML) over every run's tiles
template <class T>
void launch_ampere_batch(const StepArgs<T>* a, const BatchGrid& bg, bool filt_J, int pt_taps, size_t amp_smem,
                         cudaStream_t s);
// plasma rows entering through the +z plane of every run, then the runs' particle and chunk counts
template <class T>
void launch_inject_batch(const StepArgs<T>* a, const BatchGrid& bg, cudaStream_t s);
// the test beams of every run with one (blockIdx.y: run; beam_blocks: blocks of 128 particles of the largest)
template <class T>
void launch_beam_push_batch(const StepArgs<T>* a, int nruns, int beam_blocks, cudaStream_t s);
// filter taps and shared-memory sizes the batched field kernels need (the same as a single run's)
template <class T>
FilterTaps<T> filter_taps(const FilterSpec& fs);
template <class T>
int filter_taps_class(const FilterTaps<T>& ft);
template <class T>
size_t tile_smem_bytes(const TileMaps& tm, int H);

}  // namespace picgb
