// C ABI of the GB300 boosted-frame PIC library (include/pic.h): context,
// device memory through the caller's allocator, host-side scheduling of the
// per-step launches (all arithmetic of the step runs in the kernels of
// pic_fields.cu, pic_particles.cu and pic_aux.cu).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "../../include/pic.h"
#include "pic_3d.h"
#include "pic_batch.h"
#include "pic_common.cuh"

namespace picgb {
int push_occupancy(int order, bool dbl, int smem_nodes);
}

using namespace picgb;

namespace {

struct HostGeom {
  double dx, dz, dt, gamma, beta, a2, b2, dt_cfl;
  int guard, gx_lo, gx_hi, gz_lo, gz_hi, ld;
};

double lab_density_h(const pic_plasma& p, double zl) {
  if (zl < p.z_start_lab) return 0.0;
  double r = zl - p.z_start_lab;
  if (p.ramp_lab > 0.0 && r < p.ramp_lab) return p.n0 * r / p.ramp_lab;
  double pe = p.ramp_lab + p.length_lab;
  if (p.length_lab > 0.0 && r >= pe) return 0.0;
  return p.n0;
}

// 2D stability limit of the tunable solver restricted to d/dy = 0 (Eq. cfl), Friedman factor (Sec. 4.3)
double cfl_2d(double a, double g, double dx, double dz, double theta) {
  double kx = 1.0 / (dx * dx), kz = 1.0 / (dz * dz);
  double mx = kx > kz ? kx : kz;
  double t = (a - 4.0 * g) * (kx + kz);
  if (t > mx) mx = t;
  return 1.0 / std::sqrt(mx) / kC * std::sqrt((2.0 + theta) / (2.0 + 3.0 * theta));
}

}  // namespace

struct SimBase {
  virtual ~SimBase() {}
};

struct pic_ctx {
  pic_config cfg;
  HostGeom hg;
  cudaStream_t stream = nullptr;
  pic_alloc_fn alloc = nullptr;
  pic_free_fn freef = nullptr;
  void* user = nullptr;
  struct A { void* p; size_t n; };
  std::vector<A> allocs;
  std::string err;
  int status = PIC_OK;
  int64_t launches = 0;
  std::unique_ptr<SimBase> sim;
  std::unique_ptr<picgb::Sim3Api> s3;   // 3D and 1D contexts

  void* dalloc(size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (alloc) p = alloc(bytes, (void*)stream, user);
    else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
    if (!p) return nullptr;
    allocs.push_back({p, bytes});
    cudaMemsetAsync(p, 0, bytes, stream);
    return p;
  }
  void release_all() {
    for (auto& a : allocs) {
      if (freef) freef(a.p, a.n, (void*)stream, user);
      else cudaFree(a.p);
    }
    allocs.clear();
  }
  int fail(int code, const std::string& m) {
    if (status == PIC_OK) { status = code; err = m; }
    return code;
  }
};

namespace {

// particle shape (Sec. 2.3): linear or cubic B-spline of the distance in cells
static double host_shape(int order, double s) {
  const double a = std::fabs(s);
  if (order == 1) return a < 1.0 ? 1.0 - a : 0.0;
  if (a < 1.0) return 2.0 / 3.0 - a * a + 0.5 * a * a * a;
  if (a < 2.0) { const double t = 2.0 - a; return t * t * t / 6.0; }
  return 0.0;
}

template <class T>
struct Sim : SimBase {
  pic_ctx* c;
  GridP g;
  FieldPtrs<T> f{};
  PmlTabs pt{};
  FilterSpec fs{};
  bool friedman = false, filt_gather = false, filt_J = false;
  T* tmp = nullptr;
  Ctrl* ctrl = nullptr;
  Ctrl* hmirror = nullptr;     // pinned
  double* hstats = nullptr;    // pinned: the diagnostics' sums and a copy of the control block
  TileMaps tmaps{};
  // particles
  Particles<T> P{}, P2{};
  Chunk* chunks = nullptr;
  PushDefer pdef{};          // the push's lists for its global-memory pass
  int cap = 0, chunk_cap = 0, chunk_max = 4096, smem_nodes = 0, push_grid = 0;
  SortBufs sb{};
  int sort_every = 8;
  long long count_ub = 0;
  bool loaded = false;
  pic_plasma pl{};
  InjectP ip{};
  long long row_next = 0, row_first = 0;
  bool pairs = false;        // mixed path: electrons carry the ions of their lattice sites
  double zlo_prev = 0.0;
  // ions
  bool ions = false;
  double *ion_x = nullptr, *ion_R0 = nullptr, *ion_C = nullptr;
  // laser
  bool has_laser = false;
  LaserP lp{};
  double* ant_xs = nullptr;    // transverse antenna profile, x shape applied (nx+1)
  // beam
  Beam<T> beam{};
  double* beam_scratch = nullptr;
  // btd
  int nrows = 0;
  int* btd_idx = nullptr;
  double *btd_tp = nullptr, *btd_zp = nullptr;
  std::vector<double> h_tp;
  T* btd_out = nullptr;
  int* btd_done = nullptr;
  // bookkeeping
  long long step = 0;
  long long shifts = 0;
  int64_t sorts = 0;
  double* stats_buf = nullptr;
  double* stage = nullptr;    // (nx+1)*(nz+1) doubles
  size_t stage_n = 0;
  // timing
  bool nodal = false;   // 'momentum conserving' gather (pic_config.gather_scheme = 1)
  bool timing = false;
  int timing_which = 0;
  std::vector<cudaEvent_t> ev;
  int64_t timed_launches = 0;

  explicit Sim(pic_ctx* ctx) : c(ctx) {}
  ~Sim() override {
    for (auto e : ev) cudaEventDestroy(e);
    if (hmirror) cudaFreeHost(hmirror);
    if (hstats) cudaFreeHost(hstats);
  }

  template <class U>
  U* al(size_t n) { return (U*)c->dalloc(n * sizeof(U)); }

  int init() {
    const pic_config& cf = c->cfg;
    const HostGeom& h = c->hg;
    g.nx = cf.nx; g.nz = cf.nz; g.ld = h.ld;
    g.dx = h.dx; g.dz = h.dz; g.dt = h.dt; g.z0 = 0.0;
    g.idx = 1.0 / h.dx; g.idz = 1.0 / h.dz;
    g.dtf = (float)h.dt; g.idxf = (float)g.idx; g.idzf = (float)g.idz;
    g.gx_lo = h.gx_lo; g.gx_hi = h.gx_hi; g.gz_lo = h.gz_lo; g.gz_hi = h.gz_hi;
    g.pml = cf.pml_cells;
    g.fr_sz = 0; g.fr_fz = 0.0f;
    g.fr_u0 = (float)(-h.gamma * h.beta * kC);
    g.il_nxl = 0; g.il_ppcx = 1; g.il_ppcz = 1; g.il_kb = 0; g.z0_cells = 0;
    friedman = cf.theta != 0.0;
    filt_gather = cf.filter_gather && cf.filter_passes + cf.filter_compensate > 0;
    filt_J = cf.filter_J && cf.filter_passes + cf.filter_compensate > 0;
    fs.passes = cf.filter_passes; fs.stride = cf.filter_stride; fs.compensate = cf.filter_compensate;
    for (int q = 0; q < 4; q++) fs.strides[q] = cf.filter_stride_set[q];
    const size_t N = (size_t)(cf.nx + 1) * g.ld;
    g.cs = (long)N;
    auto grid = [&]() { return al<T>(N); };
    // 3-component blocks (component stride N): E, E-other, B, J, J-other, Bavg, gather copies, E-bar
    auto block = [&](T** dst) {
      T* b = al<T>(3 * N);
      for (int q = 0; q < 3; q++) dst[q] = b ? b + q * N : nullptr;
      return b != nullptr;
    };
    bool ok = block(f.E) && block(f.Eo) && block(f.B) && block(f.J) && block(f.Jn) && block(f.Bavg);
    if (friedman) ok = ok && block(f.Eb) && block(f.Ebn);
    if (filt_gather) ok = ok && block(f.fE) && block(f.fB);
    nodal = cf.gather_scheme == 1;
    if (nodal) ok = ok && block(f.nE) && block(f.nB);
    if (!ok) return c->fail(PIC_ENOMEM, "field allocation failed");
    if (cf.pml_cells > 0) {
      f.Byx = grid(); f.Byz = grid(); f.Eyx = grid(); f.Eyz = grid();
      if (!f.Byx || !f.Byz || !f.Eyx || !f.Eyz) return c->fail(PIC_ENOMEM, "PML allocation failed");
    }
    tmp = grid();
    if (!tmp) return c->fail(PIC_ENOMEM, "allocation failed");
    // PML tables (App. II, PR-18)
    std::vector<double> hx(6 * (cf.nx + 1)), hz(6 * (cf.nz + 1));
    auto sigma = [&](double pos, int n, double dcell) {
      int L = cf.pml_cells;
      if (L <= 0) return 0.0;
      double d = 0.0;
      if (pos < L) d = L - pos;
      if (pos > n - L) d = pos - (n - L);
      if (d <= 0.0) return 0.0;
      return cf.pml_sigma_max * kC / dcell * std::pow(d / cf.pml_delta, cf.pml_power);
    };
    auto xi = [&](double s) {
      if (cf.pml_xi_exp) return std::exp(-s * h.dt);
      return (1.0 - 0.5 * s * h.dt) / (1.0 + 0.5 * s * h.dt);
    };
    auto coef = [&](double s) { return s <= 0.0 ? h.dt : (1.0 - xi(s)) / s; };
    auto fill = [&](std::vector<double>& v, int n, double dcell) {
      for (int i = 0; i <= n; i++) {
        double si = sigma(i, n, dcell), sh = sigma(i + 0.5, n, dcell);
        v[0 * (n + 1) + i] = si; v[1 * (n + 1) + i] = sh;
        v[2 * (n + 1) + i] = xi(si); v[3 * (n + 1) + i] = xi(sh);
        v[4 * (n + 1) + i] = coef(si); v[5 * (n + 1) + i] = coef(sh);
      }
    };
    fill(hx, cf.nx, h.dx);
    fill(hz, cf.nz, h.dz);
    double* dx_t = al<double>(hx.size());
    double* dz_t = al<double>(hz.size());
    if (!dx_t || !dz_t) return c->fail(PIC_ENOMEM, "allocation failed");
    cudaMemcpyAsync(dx_t, hx.data(), hx.size() * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dz_t, hz.data(), hz.size() * 8, cudaMemcpyHostToDevice, c->stream);
    const int nx1 = cf.nx + 1, nz1 = cf.nz + 1;
    pt.sx_i = dx_t; pt.sx_h = dx_t + nx1; pt.xx_i = dx_t + 2 * nx1; pt.xx_h = dx_t + 3 * nx1;
    pt.cx_i = dx_t + 4 * nx1; pt.cx_h = dx_t + 5 * nx1;
    pt.sz_i = dz_t; pt.sz_h = dz_t + nz1; pt.xz_i = dz_t + 2 * nz1; pt.xz_h = dz_t + 3 * nz1;
    pt.cz_i = dz_t + 4 * nz1; pt.cz_h = dz_t + 5 * nz1;
    // interior index ranges, where the field kernels skip the PML branches
    auto interior = [](const std::vector<double>& v, int n, int& lo, int& hi) {
      lo = 0; hi = n;
      while (lo <= n && (v[lo] > 0.0 || v[(n + 1) + lo] > 0.0)) lo++;
      while (hi >= 0 && (v[hi] > 0.0 || v[(n + 1) + hi] > 0.0)) hi--;
    };
    interior(hx, cf.nx, pt.iin0, pt.iin1);
    interior(hz, cf.nz, pt.kin0, pt.kin1);
    ctrl = al<Ctrl>(1);
    stats_buf = al<double>(8);
    {
      const int H = (filt_gather || filt_J) ? filter_halo(fs) : 0;
      if (!make_tile_maps<T>(g, f, H, tmaps)) return c->fail(PIC_ECUDA, "TMA descriptor encoding failed");
    }
    stage_n = (size_t)nx1 * nz1;
    stage = al<double>(stage_n);
    if (!ctrl || !stats_buf || !stage) return c->fail(PIC_ENOMEM, "allocation failed");
    if (cudaMallocHost(&hmirror, sizeof(Ctrl)) != cudaSuccess) hmirror = nullptr;
    if (cudaMallocHost(&hstats, 8 * sizeof(double) + sizeof(Ctrl)) != cudaSuccess) hstats = nullptr;
    // particle tiles
    // default tile: 8 (x) by 32 (z) cells, so that a warp spans 32 consecutive z-cells
    int tx = cf.tile_x > 0 ? cf.tile_x : 8, tz = cf.tile_z > 0 ? cf.tile_z : 32;
    if (tx * tz > 1024) return c->fail(PIC_EINVAL, "tile_x * tile_z must not exceed 1024 cells");
    sb.tx = tx; sb.tz = tz;
    sb.ntx = (cf.nx + tx - 1) / tx; sb.ntz = (cf.nz + tz - 1) / tz;
    sb.R = 32;
    // the boosted-frame drift is uniform, so the cell order decays slowly
    sort_every = cf.sort_every > 0 ? cf.sort_every : 32;
    // the push's shared-memory window of a chunk: its tile plus the stencil's reach (5 cells at cubic
    // order, 3 at linear) and room for the particles to spread; no more than one cell of growth along x
    // times the row stride: padded for tile_z < 32 (tile_z + 32 nodes, congruent to tile_z modulo 32
    // banks), else unpadded with 16 cells of room. The window and the particle records then leave the L1
    // its share of the SM's 256 KB
    const int margin = 10, reach = cf.shape_order == 3 ? 5 : 3;
    smem_nodes = std::min((tx + 6 + margin) * (tz + 6 + margin), (tx + reach + 1) * (tz + (tz < 32 ? 32 : 16)));
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    push_grid = nsm * push_occupancy(cf.shape_order, sizeof(T) == 8, smem_nodes);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error during init");
  }

  void set_ptrs_for_step() {
    if (!filt_gather) {
      for (int q = 0; q < 3; q++) { f.fE[q] = f.E[q]; f.fB[q] = f.Bavg[q]; }
    }
  }

  double time_of(long long n) const { return (double)n * g.dt; }
  // frame shift of the mixed path's stored z at step n: S = beta c t / dz (cells)
  double frame_shift(long long n) const { return c->hg.beta * kC * time_of(n) / g.dz; }
  void set_frame(long long n) { frame_of(frame_shift(n), g.fr_sz, g.fr_fz); }
  double zlo() const { return g.z0 + g.gz_lo * g.dz; }
  double zhi() const { return g.z0 + g.gz_hi * g.dz; }

  long long rows_inside(double t) const {
    double y = (zhi() + c->hg.beta * kC * t) / ip.h - 0.5;
    return (long long)std::ceil(y);
  }
  long long rows_from(double t) const {
    return (long long)std::ceil((zlo() + c->hg.beta * kC * t) / ip.h - 0.5);
  }
  // particle ids of rows [a, b): row * nxl + column (FP64 path) or (row << kb) | column (mixed)
  bool ids_fit(long long a, long long b) const {
    if (a < 0) return false;
    if (CellPos<T>::value) return b <= (1LL << (32 - g.il_kb));
    return b * (long long)ip.nxl <= (1LL << 32);
  }
  bool row_has_density(long long m) const {
    double zlat = (m + 0.5) * ip.h;
    return c->hg.gamma * lab_density_h(pl, c->hg.gamma * zlat) > 0.0;
  }

  int load_plasma(const pic_plasma* p) {
    if (loaded) return c->fail(PIC_ESTATE, "plasma already loaded");
    pl = *p;
    set_frame(step);
    const pic_config& cf = c->cfg;
    const HostGeom& h = c->hg;
    if (pl.ppc_x < 1 || pl.ppc_z < 1) return c->fail(PIC_EINVAL, "ppc must be >= 1");
    ip.h = h.dz / pl.ppc_z;
    ip.gamma = h.gamma; ip.beta = h.beta;
    ip.n0 = pl.n0; ip.z_start_lab = pl.z_start_lab; ip.ramp_lab = pl.ramp_lab; ip.length_lab = pl.length_lab;
    ip.ppc_x = pl.ppc_x; ip.ppc_z = pl.ppc_z;
    ip.nxl = (g.gx_hi - g.gx_lo) * pl.ppc_x;
    g.il_nxl = ip.nxl; g.il_ppcx = pl.ppc_x; g.il_ppcz = pl.ppc_z;
    g.il_kb = 0;
    while ((1LL << g.il_kb) < ip.nxl) g.il_kb++;
    // the mixed path lets every electron carry the lab-fixed ion of its lattice site
    // (power-of-two particles per cell: the site follows from the id by shifts)
    {
      auto pow2 = [](int v) { return v > 0 && (v & (v - 1)) == 0; };
      pairs = CellPos<T>::value && pl.ions != 0 && pl.n0 > 0.0 && pow2(pl.ppc_x) && pow2(pl.ppc_z);
    }
    ip.xblock = 32;
    ions = pl.ions != 0 && pl.n0 > 0.0;
    // capacity: the particle domain full of plasma plus injection headroom
    const double rows_per_step = h.beta * kC * h.dt / ip.h + 2.0;
    const long long full = (long long)(g.gz_hi - g.gz_lo + 2) * pl.ppc_z * (long long)ip.nxl;
    const long long head = (long long)(rows_per_step + 2) * ip.nxl * (sort_every + 4);
    long long want = (long long)(full * 1.05) + head + 4096;
    if (cf.moving_window) want += (long long)((cf.window_beta * kC * h.dt / ip.h + 2) * ip.nxl * (sort_every + 4));
    if (pl.n0 <= 0.0) want = 4096;
    if (want > 2000000000LL) return c->fail(PIC_EOVERFLOW, "particle capacity above 2^31");
    cap = (int)want;
    if (CellPos<T>::value && (cf.nx >= 65535 || cf.nz >= 65535)) return c->fail(PIC_EINVAL, "mixed precision needs nx, nz < 65535");
    Particles<T>* both[2] = {&P, &P2};
    for (Particles<T>* q : both) {
      bool okp;
      if (CellPos<T>::value) {
        q->cell = al<uint32_t>(cap); q->ox = al<float>(cap); q->oz = al<float>(cap);
        okp = q->cell && q->ox && q->oz;
      } else {
        q->x = al<double>(cap); q->z = al<double>(cap);
        okp = q->x && q->z;
      }
      q->ux = al<T>(cap); q->uy = al<T>(cap); q->uz = al<T>(cap); q->w = al<T>(cap);
      q->id = al<uint32_t>(cap);
      if (!okp || !q->ux || !q->uy || !q->uz || !q->w || !q->id) return c->fail(PIC_ENOMEM, "particle allocation failed");
    }
    const int ntiles = sb.ntx * sb.ntz;
    const int xblocks = (g.gx_hi - g.gx_lo + ip.xblock - 1) / ip.xblock;
    const int inj_chunks = xblocks * 4;
    // the initial load injects every row at once, in chunks of 8 rows by one x-block
    const long long init_rows = std::max(0LL, rows_inside(time_of(step)) - rows_from(time_of(step)));
    const long long init_chunks = (long long)xblocks * ((init_rows + 7) / 8);
    chunk_cap = (int)std::max((long long)(2 * ntiles + cap / chunk_max), init_chunks) + inj_chunks * (sort_every + 4) +
                4096;
    chunks = al<Chunk>(chunk_cap);
    pdef.ovf_cap = chunk_cap;
    pdef.defer_cap = std::max(cap / 16, 65536);
    pdef.ovf = al<int>(pdef.ovf_cap);
    pdef.defer = al<int2>(pdef.defer_cap);
    if (!pdef.ovf || !pdef.defer) return c->fail(PIC_ENOMEM, "push list allocation failed");
    if (ntiles > 1024 * 1024) return c->fail(PIC_EINVAL, "too many particle tiles; enlarge tile_x/tile_z");
    const size_t ncells = (size_t)ntiles * sb.tx * sb.tz;
    sb.cell_cnt = al<int>(ncells);
    sb.cell_start = al<int>(ncells);
    sb.tile_cnt = al<int>(ntiles + 1);
    sb.tile_start = al<int>(ntiles + 1);
    sb.key = al<int>(cap);
    sb.slot = al<int>(cap);
    sb.dest = al<int>(cap);
    sb.scan_tmp = al<int>(1024 + (ntiles + 1023) / 1024);
    if (!chunks || !sb.cell_cnt || !sb.cell_start || !sb.tile_cnt || !sb.tile_start || !sb.key || !sb.slot ||
        !sb.dest || !sb.scan_tmp)
      return c->fail(PIC_ENOMEM, "sort allocation failed");
    if (ions) {
      ion_x = al<double>(cf.nx + 1);
      ion_R0 = al<double>(cf.nz + 1); ion_C = al<double>(cf.nz + 1);
      if (!ion_x || !ion_R0 || !ion_C) return c->fail(PIC_ENOMEM, "allocation failed");
      // transverse lattice profile sum_a S(X_a - i)
      std::vector<double> xp(cf.nx + 1, 0.0);
      for (int a = 0; a < ip.nxl; a++) {
        double X = ((g.gx_lo + (a + 0.5) / pl.ppc_x) * g.dx) / g.dx;
        int fx = (int)std::floor(X);
        for (int i = fx - 2; i <= fx + 3; i++) {
          if (i < 0 || i > cf.nx) continue;
          xp[i] += host_shape(cf.shape_order, X - i);
        }
      }
      cudaMemcpyAsync(ion_x, xp.data(), xp.size() * 8, cudaMemcpyHostToDevice, c->stream);
    }
    // initial rows (PR-12)
    const double t = time_of(step);
    long long m_end = rows_inside(t);
    long long m_beg = rows_from(t);
    row_first = m_beg;
    row_next = m_end;
    zlo_prev = zlo();
    if (pl.n0 > 0.0) {
      long long a = m_beg, b = m_end;
      while (a < b && !row_has_density(a)) a++;
      while (b > a && !row_has_density(b - 1)) b--;
      if (b > a) {
        if (!ids_fit(a, b)) return c->fail(PIC_EOVERFLOW, "plasma rows exceed the 32-bit particle id space");
        ip.m_beg = a; ip.m_end = b; ip.t = t; ip.rblock = 8;
        if ((b - a) * (long long)ip.nxl > cap) return c->fail(PIC_EOVERFLOW, "initial plasma exceeds capacity");
        launch_inject<T>(g, P, chunks, ctrl, ip, cap, chunk_cap, c->stream);
        c->launches += 2;
        count_ub = (b - a) * (long long)ip.nxl;
        do_sort();
      }
    }
    // test beam
    if (p->beam_n > 0) {
      if (!p->beam_x || !p->beam_z || !p->beam_ux || !p->beam_uy || !p->beam_uz) return c->fail(PIC_EINVAL, "beam arrays missing");
      const int n = (int)p->beam_n;
      beam.n = n;
      beam.x = al<double>(n); beam.z = al<double>(n); beam.ux = al<T>(n); beam.uy = al<T>(n); beam.uz = al<T>(n);
      beam.tc = al<double>(n); beam.zf0 = al<double>(n); beam.uxb = al<T>(n); beam.uyb = al<T>(n); beam.uzb = al<T>(n);
      beam.flag = al<int>(n);
      if (p->beam_self) {
        // self-consistent beam: weights (per unit length along y), converted to the path's type
        if (!p->beam_w) return c->fail(PIC_EINVAL, "beam_self needs beam_w");
        std::vector<T> wv(n);
        for (int q = 0; q < n; q++) wv[q] = T(p->beam_w[q]);
        beam.w = al<T>(n);
        if (!beam.w) return c->fail(PIC_ENOMEM, "beam allocation failed");
        cudaMemcpyAsync(beam.w, wv.data(), sizeof(T) * n, cudaMemcpyHostToDevice, c->stream);
        cudaStreamSynchronize(c->stream);
        beam.self = 1;
      }
      beam_scratch = al<double>(4);
      double* lab = al<double>(5 * (size_t)n);
      if (!beam.x || !beam.flag || !lab || !beam_scratch) return c->fail(PIC_ENOMEM, "beam allocation failed");
      const double* srcs[5] = {p->beam_x, p->beam_z, p->beam_ux, p->beam_uy, p->beam_uz};
      for (int q = 0; q < 5; q++) cudaMemcpyAsync(lab + (size_t)q * n, srcs[q], 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
      cudaStreamSynchronize(c->stream);   // host arrays are only valid during the call
      launch_beam_init<T>(beam, lab, lab + n, lab + 2 * (size_t)n, lab + 3 * (size_t)n, lab + 4 * (size_t)n, p->beam_t_lab,
                          p->beam_z_plane_lab, h.gamma, h.beta, time_of(step), beam_scratch, c->stream);
      c->launches += 3;
    }
    loaded = true;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in load_plasma");
  }

  void do_sort() {
    launch_sort<T>(g, P, P2, sb, chunks, ctrl, cap, chunk_max, chunk_cap, c->stream);
    c->launches += 8;
    std::swap(P, P2);
    sorts++;
    if (hmirror) cudaMemcpyAsync(&hmirror->count, &ctrl->count, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  }

  int set_laser(const pic_laser* l) {
    lp.lambda0 = l->lambda0; lp.a0 = l->a0; lp.w0 = l->w0; lp.tau = l->tau_fwhm; lp.t_peak = l->t_peak;
    lp.x_center = l->x_center; lp.phase = l->phase; lp.z_antenna = l->z_antenna; lp.beta_s = l->beta_s;
    lp.gamma = c->hg.gamma; lp.beta = c->hg.beta;
    if (!(l->lambda0 > 0) || !(l->w0 > 0) || !(l->tau_fwhm > 0)) return c->fail(PIC_EINVAL, "laser lambda0, w0, tau must be > 0");
    // transverse Gaussian of the emitted field on the nodes inside the particle
    // domain, spread by the x shape: xs[i] = sum_d S(d) G(i + d)
    const pic_config& cf = c->cfg;
    std::vector<double> G(cf.nx + 1, 0.0), xs(cf.nx + 1, 0.0);
    for (int i = g.gx_lo; i <= g.gx_hi && i <= cf.nx; i++) {
      const double dxr = i * g.dx - lp.x_center;
      G[i] = std::exp(-dxr * dxr / (lp.w0 * lp.w0));
    }
    for (int i = 0; i <= cf.nx; i++)
      for (int d = -2; d <= 2; d++) {
        const int ia = i + d;
        const double wx = host_shape(cf.shape_order, (double)d);
        if (ia >= 0 && ia <= cf.nx && wx != 0.0) xs[i] += G[ia] * wx;
      }
    if (!ant_xs) ant_xs = al<double>(cf.nx + 1);
    if (!ant_xs) return c->fail(PIC_ENOMEM, "allocation failed");
    cudaMemcpyAsync(ant_xs, xs.data(), xs.size() * 8, cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    has_laser = true;
    return PIC_OK;
  }

  // the antenna of one step [t0, t1] (Sec. 3.1.2): K_y = -2 eps0 c E_emit with
  // E_emit = (1 - beta_s) / ((1 + beta) gamma) g(x, (1 - beta_s) t / ((1 + beta) gamma))
  // evaluated at the mid time; false when the antenna is outside the particle domain
  bool antenna_step(double t0, double t1, AntennaStep& a) const {
    const int order = c->cfg.shape_order;
    const double za0 = lp.z_antenna + lp.beta_s * kC * t0;
    const double za1 = lp.z_antenna + lp.beta_s * kC * t1;
    const double zlo = g.z0 + g.gz_lo * g.dz, zhi = g.z0 + g.gz_hi * g.dz;
    if (za0 < zlo || za0 >= zhi || za1 < zlo || za1 >= zhi) return false;
    const double om = 2.0 * kPi * kC / lp.lambda0;
    const double E0 = lp.a0 * kMe * kC * om / kQe;
    const double dop = (1.0 + lp.beta) * lp.gamma;
    const double sl = (1.0 - lp.beta_s) * (0.5 * (t0 + t1)) / dop;
    const double sig = lp.tau / (2.0 * std::sqrt(std::log(2.0)));
    const double u = sl - lp.t_peak;
    a.amp = -2.0 * kEps0 * kC * (1.0 - lp.beta_s) / dop * E0 * std::exp(-u * u / (2.0 * sig * sig)) *
            std::sin(om * u + lp.phase);
    const double Z0 = (za0 - g.z0) / g.dz, Z1 = (za1 - g.z0) / g.dz;
    const int fz = (int)std::floor(Z0 < Z1 ? Z0 : Z1);
    a.k0 = fz - 3;
    for (int j = 0; j < 8; j++) {
      const int k = a.k0 + j;
      a.wz[j] = 0.5 * (host_shape(order, Z0 - k) + host_shape(order, Z1 - k)) / g.dz;
    }
    return true;
  }

  void btd_range(double ta, double tb, int& r0, int& r1) const {
    r0 = (int)(std::lower_bound(h_tp.begin(), h_tp.end(), ta) - h_tp.begin());
    r1 = (int)(std::lower_bound(h_tp.begin(), h_tp.end(), tb) - h_tp.begin());
  }

  void btd(int post) {
    if (nrows == 0) return;
    const double tn = time_of(step);
    int r0, r1;
    btd_range(tn, time_of(step + 1), r0, r1);
    if (r1 > r0) {
      launch_btd<T>(g, f, 0, post, r0, r1, btd_idx, btd_tp, btd_zp, tn, c->hg.gamma, c->hg.beta, btd_out, btd_done, c->stream);
      c->launches++;
    }
    const double ta = tn - 0.5 * g.dt;
    btd_range(ta, ta + g.dt, r0, r1);
    if (r1 > r0) {
      launch_btd<T>(g, f, 1, post, r0, r1, btd_idx, btd_tp, btd_zp, ta, c->hg.gamma, c->hg.beta, btd_out, btd_done, c->stream);
      c->launches++;
    }
  }

  void window_shift() {
    const pic_config& cf = c->cfg;
    if (!cf.moving_window) return;
    const double t = time_of(step);
    long long want = (long long)std::floor(cf.window_beta * kC * t / g.dz);
    long long sh = want - shifts;
    if (sh <= 0) return;
    for (int q = 0; q < 3; q++) {
      launch_shift<T>(g, f.E[q], tmp, (int)sh, EX + q, c->stream);
      launch_shift<T>(g, f.Eo[q], tmp, (int)sh, EX + q, c->stream);
      launch_shift<T>(g, f.B[q], tmp, (int)sh, BX + q, c->stream);
      if (friedman) launch_shift<T>(g, f.Eb[q], tmp, (int)sh, EX + q, c->stream);
      c->launches += friedman ? 4 : 3;
    }
    if (cf.pml_cells > 0) {
      T* arrs[4] = {f.Byx, f.Byz, f.Eyx, f.Eyz};
      const int comps[4] = {BY, BY, EY, EY};
      for (int q = 0; q < 4; q++) { launch_shift<T>(g, arrs[q], tmp, (int)sh, comps[q], c->stream); c->launches++; }
    }
    if (loaded && chunks) {
      launch_shift_chunks(chunks, ctrl, (int)sh, chunk_cap, c->stream);
      launch_shift_particles<T>(g, P, ctrl, cap, (int)sh, c->stream);
      c->launches += CellPos<T>::value ? 2 : 1;
    }
    shifts = want;
    g.z0 = (double)want * g.dz;
    g.z0_cells = (int)want;
  }

  void refresh_count_bound(long long add) {
    if (count_ub + add <= cap) return;
    // read the device count after a synchronisation; compact if needed
    cudaStreamSynchronize(c->stream);
    Ctrl hc;
    cudaMemcpy(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    count_ub = hc.count;
    if (count_ub + add > cap) {
      do_sort();
      cudaStreamSynchronize(c->stream);
      cudaMemcpy(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
      count_ub = hc.count;
    }
  }

  int one_step() {
    const pic_config& cf = c->cfg;
    const HostGeom& h = c->hg;
    const double tn = time_of(step), tn1 = time_of(step + 1);
    set_frame(step);
    window_shift();
    set_ptrs_for_step();
    btd(0);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto tstart = [&](int which) {
      if (timing && timing_which == which) {
        cudaEventCreate(&e0); cudaEventCreate(&e1);
        cudaEventRecord(e0, c->stream);
      }
    };
    auto tstop = [&](int which) {
      if (timing && timing_which == which && e0) {
        cudaEventRecord(e1, c->stream);
        ev.push_back(e0); ev.push_back(e1);
        e0 = e1 = nullptr;
        timed_launches++;
      }
    };
    // 1. Faraday + Friedman + PML-B (B^{n-1/2} -> B^{n+1/2}, Bavg), fused with the gather filter of E^n
    //    where the filter allows
    tstart(1);
    const bool fused = launch_faraday_fused<T>(g, f, pt, h.a2, h.b2, cf.theta, friedman, fs, filt_gather, tmaps,
                                               ctrl, c->stream);
    if (!fused) launch_faraday<T>(g, f, pt, h.a2, h.b2, cf.theta, friedman, c->stream);
    // 2. gather copies (interpolated to the nodes for the 'momentum conserving' gather): B_avg, and E^n
    //    unless the fused kernel filtered it
    launch_filter_fields<T>(g, f, fs, filt_gather, tmaps, ctrl, c->stream, fused ? 3 : 0);
    if (nodal) launch_nodal<T>(g, f, c->stream);
    tstop(1);
    c->launches += 1 + (filt_gather ? 1 : 0) + (nodal ? 1 : 0);
    // ion rows live during this step: those inside the particle domain at t^n
    long long mlo = std::max(row_first, (long long)std::ceil((zlo_prev + h.beta * kC * tn) / ip.h - 0.5));
    if (step == 0) mlo = row_first;
    // 3. particles
    if (loaded && cap > 0) {
      tstart(0);
      int fr1_sz;
      float fr1_fz;
      frame_of(frame_shift(step + 1), fr1_sz, fr1_fz);
      launch_push<T>(g, f, P, chunks, ctrl, cf.shape_order, push_grid, smem_nodes, sb.tz, -kQe, kMe, c->hg.gamma,
                     c->hg.beta,
                     fr1_sz, fr1_fz, (pairs && ions) ? 1 : 0, (int)mlo, nodal ? 1 : 0, pdef, c->stream);
      tstop(0);
      c->launches += 2;
    }
    set_frame(step + 1);   // the particles now hold their t^{n+1} positions
    if (beam.n > 0) {
      launch_beam_push<T>(g, f, beam, cf.shape_order, tn, tn1, nodal ? 1 : 0, beam_scratch, c->stream);
      c->launches++;
    }
    // 4. antenna
    AntennaStep ast;
    if (has_laser && antenna_step(tn, tn1, ast)) {
      launch_antenna<T>(g, f.J[1], ant_xs, ast, c->stream);
      c->launches++;
    }
    // 5. ion column current (unless every electron carries its ion)
    double ion_coef = 0.0;
    const bool column = ions && loaded && !pairs;
    if (column) {
      launch_ion_column(g, mlo, row_next, tn, tn1, ip, cf.shape_order, ion_C, c->stream);
      c->launches += 1;
      ion_coef = -kQe / (g.dx * g.dt);
    }
    // 6-7. current filter + Ampere + PML-E
    tstart(1);
    launch_ampere<T>(g, f, pt, fs, filt_J, column ? ion_x : nullptr, ion_C, ion_coef, tmaps, ctrl, c->stream);
    tstop(1);
    c->launches++;
    for (int q = 0; q < 3; q++) {
      std::swap(f.E[q], f.Eo[q]);
      std::swap(f.J[q], f.Jn[q]);
      if (friedman) std::swap(f.Eb[q], f.Ebn[q]);
    }
    set_ptrs_for_step();
    btd(1);
    zlo_prev = zlo();
    // 8. plasma rows entering through z_hi
    if (loaded && pl.n0 > 0.0) {
      long long m_end = rows_inside(tn1);
      long long a = row_next, b = m_end;
      if (b > row_next) row_next = b;
      while (a < b && !row_has_density(a)) a++;
      while (b > a && !row_has_density(b - 1)) b--;
      if (b > a) {
        long long add = (b - a) * (long long)ip.nxl;
        refresh_count_bound(add);
        if (count_ub + add > cap) return c->fail(PIC_EOVERFLOW, "particle capacity exceeded");
        if (!ids_fit(a, b)) return c->fail(PIC_EOVERFLOW, "plasma rows exceed the 32-bit particle id space");
        ip.m_beg = a; ip.m_end = b; ip.t = tn1; ip.rblock = 4;
        launch_inject<T>(g, P, chunks, ctrl, ip, cap, chunk_cap, c->stream);
        c->launches += 2;
        count_ub += add;
      }
    }
    step++;
    if (loaded && cap > 0 && step % sort_every == 0) do_sort();
    return PIC_OK;
  }

  // ---- batched (ensemble) stepping ---------------------------------------------------------------------
  // A run the batched ensemble step carries: plasma loaded, the Yee-located gather, no lab samples, no
  // moving window (those steps keep the per-run launches); a test beam rides along.
  bool batchable() const {
    const pic_config& cf = c->cfg;
    return loaded && cap > 0 && !nodal && nrows == 0 && !cf.moving_window && tmaps.ok;
  }
  // upper bounds of the per-step work of the batched kernels that do not run a fixed grid
  int inj_xblocks() const { return (g.gx_hi - g.gx_lo + ip.xblock - 1) / ip.xblock; }
  int inj_rblocks_max() const { return (int)std::ceil(c->hg.beta * kC * g.dt / ip.h) / 4 + 2; }
  long long ion_rows_max() const { return (long long)(g.gz_hi - g.gz_lo + 8) * pl.ppc_z + 16; }

  // The host decisions of one step, in the order of one_step, written into the run's argument block of a
  // batched launch instead of launching; then the step's bookkeeping. sort_after: the run sorts after this
  // step (its sort is launched after the batched kernels). Returns PIC_OK or the error of a step that the
  // batched kernels cannot carry.
  int plan_step(StepArgs<T>& a, bool& sort_after) {
    const pic_config& cf = c->cfg;
    const HostGeom& h = c->hg;
    const double tn = time_of(step), tn1 = time_of(step + 1);
    set_frame(step);
    set_ptrs_for_step();
    a.g = g;
    a.f = f;
    a.pt = pt;
    a.far = faraday_coefs<T>(h.a2, h.b2, cf.theta);
    a.ft = filter_taps<T>(fs);
    a.filt_gather = filt_gather;
    a.filt_J = filt_J;
    a.tm = tmaps;
    a.mapE = tmaps.Ebase[0] == (const void*)f.E[0] ? 0 : 1;
    a.mapJ = tmaps.Jbase[0] == (const void*)f.J[0] ? 0 : 1;
    a.mapEb = tmaps.Ebbase[0] == (const void*)f.Eb[0] ? 0 : 1;
    field_tiles(g, a.tiles_k, a.tiles_i);
    // ion rows live during this step: those inside the particle domain at t^n
    long long mlo = std::max(row_first, (long long)std::ceil((zlo_prev + h.beta * kC * tn) / ip.h - 0.5));
    if (step == 0) mlo = row_first;
    int fr1_sz;
    float fr1_fz;
    frame_of(frame_shift(step + 1), fr1_sz, fr1_fz);
    a.pc = push_const(g, -kQe, kMe, c->hg.gamma, fr1_sz, fr1_fz, (pairs && ions) ? 1 : 0, (int)mlo);
    a.p = P;
    a.chunks = chunks;
    a.ctrl = ctrl;
    a.pd = pdef;
    a.push_on = 1;
    set_frame(step + 1);
    // the test beam, pushed with the same fields after the plasma
    a.beam_on = beam.n > 0;
    a.beam = beam;
    a.beam_order = cf.shape_order;
    a.beam_tn = tn;
    a.beam_tn1 = tn1;
    a.beam_acc = beam_scratch;
    a.ant_on = has_laser && antenna_step(tn, tn1, a.ast);
    a.ant_xs = ant_xs;
    const bool column = ions && loaded && !pairs;
    a.ion_on = column;
    a.ion_order = cf.shape_order;
    a.ion_mlo = mlo;
    a.ion_mhi = row_next;
    a.ion_t0 = tn;
    a.ion_t1 = tn1;
    a.ion_coef = column ? -kQe / (g.dx * g.dt) : 0.0;
    a.ion_C = ion_C;
    a.ion_x = ion_x;
    if (column && row_next - mlo > ion_rows_max()) return c->fail(PIC_EOVERFLOW, "batched step: ion rows above bound");
    for (int q = 0; q < 3; q++) {
      std::swap(f.E[q], f.Eo[q]);
      std::swap(f.J[q], f.Jn[q]);
      if (friedman) std::swap(f.Eb[q], f.Ebn[q]);
    }
    set_ptrs_for_step();
    zlo_prev = zlo();
    a.inj_on = 0;
    a.ip = ip;
    if (loaded && pl.n0 > 0.0) {
      long long m_end = rows_inside(tn1);
      long long ra = row_next, rb = m_end;
      if (rb > row_next) row_next = rb;
      while (ra < rb && !row_has_density(ra)) ra++;
      while (rb > ra && !row_has_density(rb - 1)) rb--;
      if (rb > ra) {
        long long add = (rb - ra) * (long long)ip.nxl;
        refresh_count_bound(add);
        if (count_ub + add > cap) return c->fail(PIC_EOVERFLOW, "particle capacity exceeded");
        if (!ids_fit(ra, rb)) return c->fail(PIC_EOVERFLOW, "plasma rows exceed the 32-bit particle id space");
        ip.m_beg = ra; ip.m_end = rb; ip.t = tn1; ip.rblock = 4;
        const int rblocks = (int)((rb - ra + ip.rblock - 1) / ip.rblock);
        if (rblocks > inj_rblocks_max()) return c->fail(PIC_EOVERFLOW, "batched step: inflow rows above bound");
        a.ip = ip;
        a.inj_on = 1;
        a.inj_xblocks = inj_xblocks();
        a.cap = cap;
        a.chunk_cap = chunk_cap;
        a.add_count = (int)add;
        a.add_chunks = a.inj_xblocks * rblocks;
        count_ub += add;
      }
    }
    step++;
    sort_after = loaded && cap > 0 && step % sort_every == 0;
    return PIC_OK;
  }

  int run(int n) {
    for (int i = 0; i < n; i++) {
      int r = one_step();
      if (r != PIC_OK) return r;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return c->fail(PIC_ECUDA, std::string("CUDA error in pic_step: ") + cudaGetErrorString(e));
    return PIC_OK;
  }

  int btd_set(const pic_btd_req* r) {
    const int n = (int)r->n_rows;
    if (n <= 0 || !r->z_lab || !r->t_lab) return c->fail(PIC_EINVAL, "empty lab-sample request");
    const double ga = c->hg.gamma, be = c->hg.beta;
    std::vector<double> tp(n), zp(n);
    std::vector<int> idx(n);
    for (int i = 0; i < n; i++) {
      tp[i] = ga * (r->t_lab[i] - be * r->z_lab[i] / kC);
      zp[i] = ga * (r->z_lab[i] - be * kC * r->t_lab[i]);
      idx[i] = i;
    }
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return tp[a] < tp[b]; });
    std::vector<double> stp(n), szp(n);
    for (int i = 0; i < n; i++) { stp[i] = tp[idx[i]]; szp[i] = zp[idx[i]]; }
    nrows = n;
    h_tp = stp;
    btd_idx = al<int>(n); btd_tp = al<double>(n); btd_zp = al<double>(n);
    btd_out = al<T>((size_t)n * 6 * (g.nx + 1));
    btd_done = al<int>(2 * (size_t)n);
    if (!btd_idx || !btd_tp || !btd_zp || !btd_out || !btd_done) return c->fail(PIC_ENOMEM, "lab-sample allocation failed");
    cudaMemcpyAsync(btd_idx, idx.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(btd_tp, stp.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(btd_zp, szp.data(), 8 * (size_t)n, cudaMemcpyHostToDevice, c->stream);
    cudaStreamSynchronize(c->stream);
    return PIC_OK;
  }

  int btd_get(pic_btd_out* o) {
    if (nrows == 0) return c->fail(PIC_ESTATE, "no lab-sample request registered");
    const size_t n = (size_t)nrows * 6 * (g.nx + 1);
    cudaStreamSynchronize(c->stream);
    cudaMemcpyKind k = o->on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (o->data) cudaMemcpy(o->data, btd_out, n * sizeof(T), k);
    std::vector<int> d(2 * (size_t)nrows);
    cudaMemcpy(d.data(), btd_done, d.size() * 4, cudaMemcpyDeviceToHost);
    if (o->done) cudaMemcpy(o->done, btd_done, d.size() * 4, k);
    int64_t full = 0;
    for (int i = 0; i < nrows; i++) full += (d[2 * i] && d[2 * i + 1]) ? 1 : 0;
    o->n_rows_filled = full;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in lab-sample copy");
  }

  int get_field(int comp, double* dst, int on_device) {
    set_ptrs_for_step();
    const size_t n = stage_n;
    if (comp >= PIC_EX && comp <= PIC_JZ) {
      const T* src = comp < 3 ? f.E[comp] : comp < 6 ? f.B[comp - 3] : f.Jn[comp - 6];
      launch_convert<T>(src, stage, g, c->stream);
    } else if (comp == PIC_RHO) {
      cudaMemsetAsync(stage, 0, n * 8, c->stream);
      if (loaded) launch_rho<T>(g, P, ctrl, cap, c->cfg.shape_order, -kQe, stage, c->stream);
      if (ions && loaded) {
        const double t = time_of(step);
        long long mlo = std::max(row_first, (long long)std::ceil((zlo_prev + c->hg.beta * kC * t) / ip.h - 0.5));
        if (step == 0) mlo = row_first;
        launch_ion_rows(g, mlo, row_next, t, ip, c->cfg.shape_order, ion_R0, c->stream);
        launch_ion_rho(g, ion_x, ion_R0, kQe / (g.dx * g.dz), stage, c->stream);
      }
    } else {
      return c->fail(PIC_EINVAL, "unknown component");
    }
    cudaStreamSynchronize(c->stream);
    cudaMemcpy(dst, stage, n * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in get_field");
  }

  int get_rho_noalloc(double* dst) {
    long long mlo = row_first;
    if (ions && loaded && step > 0) {
      const double t = time_of(step);
      mlo = std::max(row_first, (long long)std::ceil((zlo_prev + c->hg.beta * kC * t) / ip.h - 0.5));
    }
    cudaError_t why = cudaSuccess;
    int kernels = 0;
    int r = launch_rho_noalloc<T>(g, P, ctrl, loaded ? cap : 0, c->cfg.shape_order, ions && loaded, mlo, row_next,
                                  time_of(step), ip, ion_x, dst, c->stream, &why, &kernels);
    c->launches += kernels;
    if (r == 1) return c->fail(PIC_EINVAL, "pic_get_rho_noalloc: nz exceeds PIC_NOALLOC_MAX_NZ");
    if (r == 2)
      return c->fail(PIC_ECUDA, std::string("pic_get_rho_noalloc: cudaGetSymbolAddress of the scratch failed: ") +
                                    cudaGetErrorString(why));
    if (r == 3)
      return c->fail(PIC_ECUDA, std::string("pic_get_rho_noalloc: kernel launch failed: ") + cudaGetErrorString(why));
    return PIC_OK;
  }

  // the frozen beam's self-field (Sec. 3.1.1, PR-27), solved on the device and added to E and B_y
  int beam_self_field() {
    if (beam.n <= 0 || !beam.self) return c->fail(PIC_ESTATE, "pic_beam_self_field: no self-consistent test beam");
    const pic_config& cf = c->cfg;
    if (cf.nx < 2 || cf.nz < 2) return c->fail(PIC_EINVAL, "pic_beam_self_field: grid too small");
    double* tmp = al<double>(stage_n);
    double* tabx = al<double>(2 * (size_t)cf.nx);
    double* tabz = al<double>(2 * (size_t)cf.nz);
    if (!tmp || !tabx || !tabz) return c->fail(PIC_ENOMEM, "pic_beam_self_field: scratch allocation failed");
    std::vector<double> tx(2 * (size_t)cf.nx), tz(2 * (size_t)cf.nz);
    for (int t = 0; t < 2 * cf.nx; t++) tx[t] = std::sin(kPi * t / cf.nx);
    for (int t = 0; t < 2 * cf.nz; t++) tz[t] = std::sin(kPi * t / cf.nz);
    cudaMemcpyAsync(tabx, tx.data(), tx.size() * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(tabz, tz.data(), tz.size() * 8, cudaMemcpyHostToDevice, c->stream);
    double v = 0.0;
    cudaMemcpyAsync(&v, beam_scratch + 2, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
    const double gv2 = 1.0 / (1.0 - (v / kC) * (v / kC));
    set_ptrs_for_step();
    launch_beam_self_field<T>(g, f, beam, cf.shape_order, beam_scratch, gv2, stage, tmp, tabx, tabz, c->stream);
    c->launches += 18;
    cudaStreamSynchronize(c->stream);
    free_last(3);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in pic_beam_self_field");
  }

  int set_field(int comp, const double* src) {
    if (comp < PIC_EX || comp > PIC_BZ) return c->fail(PIC_EINVAL, "only E and B can be set");
    cudaMemcpyAsync(stage, src, stage_n * 8, cudaMemcpyHostToDevice, c->stream);
    launch_convert_back<T>(stage, comp < 3 ? f.E[comp] : f.B[comp - 3], g, c->stream);
    cudaStreamSynchronize(c->stream);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in set_field");
  }

  int get_particles(int species, double* x, double* z, double* ux, double* uy, double* uz, double* w, uint32_t* id,
                    int32_t* flags, int64_t* count) {
    cudaStreamSynchronize(c->stream);
    if (species == PIC_BEAM) {
      const int n = beam.n;
      if (!x) { *count = n; return PIC_OK; }
      if (*count < n) return c->fail(PIC_EINVAL, "output capacity too small");
      std::vector<T> tu(n);
      std::vector<int> fl(n);
      if (n > 0) {
        cudaMemcpy(x, beam.x, 8 * (size_t)n, cudaMemcpyDeviceToHost);
        cudaMemcpy(z, beam.z, 8 * (size_t)n, cudaMemcpyDeviceToHost);
        T* srcs[3] = {beam.ux, beam.uy, beam.uz};
        double* dsts[3] = {ux, uy, uz};
        for (int q = 0; q < 3; q++) {
          cudaMemcpy(tu.data(), srcs[q], sizeof(T) * n, cudaMemcpyDeviceToHost);
          for (int j = 0; j < n; j++) dsts[q][j] = (double)tu[j];
        }
        cudaMemcpy(fl.data(), beam.flag, 4 * (size_t)n, cudaMemcpyDeviceToHost);
      }
      for (int j = 0; j < n; j++) {
        if (w) w[j] = 1.0;
        if (id) id[j] = (uint32_t)j;
        if (flags) flags[j] = fl[j];
      }
      *count = n;
      return PIC_OK;
    }
    if (species != PIC_ELECTRONS) return c->fail(PIC_EINVAL, "unknown species");
    if (!loaded || cap == 0) { *count = 0; return PIC_OK; }
    double* out6 = al<double>(6 * (size_t)cap);
    uint32_t* ido = al<uint32_t>(cap);
    int* nout = al<int>(1);
    if (!out6 || !ido || !nout) return c->fail(PIC_ENOMEM, "staging allocation failed");
    launch_compact_copy<T>(g, P, ctrl, cap, out6, ido, nout, c->stream);
    int hn = 0;
    cudaStreamSynchronize(c->stream);
    cudaMemcpy(&hn, nout, 4, cudaMemcpyDeviceToHost);
    if (!x) { *count = hn; free_last(3); return PIC_OK; }
    if (*count < hn) { free_last(3); return c->fail(PIC_EINVAL, "output capacity too small"); }
    double* dsts[6] = {x, z, ux, uy, uz, w};
    for (int q = 0; q < 6; q++)
      if (dsts[q]) cudaMemcpy(dsts[q], out6 + (size_t)q * cap, 8 * (size_t)hn, cudaMemcpyDeviceToHost);
    if (id) cudaMemcpy(id, ido, 4 * (size_t)hn, cudaMemcpyDeviceToHost);
    if (flags) for (int j = 0; j < hn; j++) flags[j] = 1;
    *count = hn;
    free_last(3);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in get_particles");
  }

  void free_last(int n) {
    for (int i = 0; i < n && !c->allocs.empty(); i++) {
      auto a = c->allocs.back();
      c->allocs.pop_back();
      cudaStreamSynchronize(c->stream);
      if (c->freef) c->freef(a.p, a.n, (void*)c->stream, c->user);
      else cudaFree(a.p);
    }
  }

  int stats(pic_stats* o) {
    set_ptrs_for_step();
    // trapping threshold (PR-19): twice the wake's Lorentz factor gamma_w = omega_laser / omega_p (lab),
    // unless the caller asks for another one
    double trap = o->trap_gamma_lab > 0.0 ? o->trap_gamma_lab : 0.0;
    if (trap == 0.0 && has_laser && loaded && pl.n0 > 0.0) {
      const double wp = std::sqrt(pl.n0 * kQe * kQe / (kEps0 * kMe));
      trap = 2.0 * (2.0 * kPi * kC / lp.lambda0) / wp;
    }
    launch_stats<T>(g, f, P, ctrl, cap, beam, c->hg.gamma, c->hg.beta, trap, stats_buf, c->stream);
    double h[8];
    Ctrl hc;
    if (hstats) {
      // both reads queued behind the reduction into pinned memory, one wait
      cudaMemcpyAsync(hstats, stats_buf, 8 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
      cudaMemcpyAsync(hstats + 8, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->stream);
      cudaStreamSynchronize(c->stream);
      std::memcpy(h, hstats, sizeof(h));
      std::memcpy(&hc, hstats + 8, sizeof(Ctrl));
    } else {
      cudaStreamSynchronize(c->stream);
      cudaMemcpy(h, stats_buf, sizeof(h), cudaMemcpyDeviceToHost);
      cudaMemcpy(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    }
    o->step = step; o->t = time_of(step);
    o->dt = g.dt; o->dx = g.dx; o->dz = g.dz; o->gamma = c->hg.gamma; o->beta = c->hg.beta;
    o->n_electrons = (int64_t)h[0];
    o->n_beam_active = (int64_t)h[1];
    o->beam_gamma_lab = h[1] > 0 ? h[2] / h[1] : 0.0;
    double var = h[1] > 0 ? h[3] / h[1] - o->beam_gamma_lab * o->beam_gamma_lab : 0.0;
    o->beam_spread = o->beam_gamma_lab > 0 ? std::sqrt(var > 0 ? var : 0) / o->beam_gamma_lab : 0.0;
    o->field_energy = h[4];
    o->gx_lo = g.gx_lo; o->gx_hi = g.gx_hi; o->gz_lo = g.gz_lo; o->gz_hi = g.gz_hi;
    o->sorts = sorts; o->overflow_chunks = hc.overflow_chunks;
    o->z0 = g.z0;
    o->trap_gamma_lab = trap;
    o->trapped_charge = kQe * h[5];
    return cudaGetLastError() == cudaSuccess ? PIC_OK : c->fail(PIC_ECUDA, "CUDA error in stats");
  }

  int sync() {
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return c->fail(PIC_ECUDA, std::string("CUDA error: ") + cudaGetErrorString(e));
    Ctrl hc;
    cudaMemcpy(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost);
    if (hc.status & ST_OVERFLOW) return c->fail(PIC_EOVERFLOW, "device capacity exceeded");
    if (hc.status & ST_NAN) return c->fail(PIC_ENAN, "non-finite particle state");
    if (hc.status & ST_OUTSIDE) return c->fail(PIC_EINVAL, "particle outside the grid");
    if (hc.status & ST_TIMEOUT) return c->fail(PIC_ETIMEOUT, "device wait timed out");
    return PIC_OK;
  }

  int kernel_timing(int enable, int which, double* ms, int64_t* nl) {
    if (enable) {
      for (auto e : ev) cudaEventDestroy(e);
      ev.clear();
      timing = true; timing_which = which; timed_launches = 0;
      return PIC_OK;
    }
    cudaStreamSynchronize(c->stream);
    double tot = 0.0;
    for (size_t i = 0; i + 1 < ev.size(); i += 2) {
      float m = 0.f;
      cudaEventElapsedTime(&m, ev[i], ev[i + 1]);
      tot += m;
    }
    if (ms) *ms = tot;
    if (nl) *nl = timed_launches;
    for (auto e : ev) cudaEventDestroy(e);
    ev.clear();
    timing = false;
    return PIC_OK;
  }
};

template <class T>
Sim<T>* S(pic_ctx* c) { return static_cast<Sim<T>*>(c->sim.get()); }

#define DISPATCH(ctx, expr)                                                  \
  ((ctx)->cfg.precision == PIC_FP64 ? S<double>(ctx)->expr : S<float>(ctx)->expr)

// The batched ensemble step: each run's host decisions fill its argument block (Sim::plan_step), one
// host-to-device copy moves all blocks, and one launch per kernel class advances every run. The argument
// blocks are double-buffered (the host fills one slot while the GPU may still read the other), and each
// slot's sequence can be captured once into a CUDA graph and replayed every step: the kernels read
// everything that changes between steps (pointers of the swapped buffers, frame shift, antenna factor,
// inflow rows) from the argument blocks, so the graph's launches never change.
template <class T>
struct BatchImpl : Batch {
  std::vector<Sim<T>*> sims;
  int n = 0;
  cudaStream_t s = nullptr;
  StepArgs<T>* dA[2] = {nullptr, nullptr};
  StepArgs<T>* hA[2] = {nullptr, nullptr};
  cudaEvent_t done[2] = {nullptr, nullptr};
  bool used[2] = {false, false};
  cudaGraphExec_t gx[2] = {nullptr, nullptr};
  bool graphs = true;
  BatchGrid bg{};
  int order = 3, pt_taps = 0, push_grid = 0, smem_nodes = 0, tile_z = 0;
  bool friedman = false, ck = false, filt_gather = false, filt_J = false, any_ion = false;
  int beam_blocks = 0;   // blocks of 128 particles of the largest test beam (0: no run has one)
  size_t filt_smem = 0, amp_smem = 0;
  size_t fused_smem = 0;   // > 0: the fused Faraday + E filter kernel serves every run
  int64_t nl = 0, nstep = 0;

  ~BatchImpl() override {
    if (s) cudaStreamSynchronize(s);
    for (int q = 0; q < 2; q++) {
      if (gx[q]) cudaGraphExecDestroy(gx[q]);
      if (done[q]) cudaEventDestroy(done[q]);
      if (hA[q]) cudaFreeHost(hA[q]);
    }
  }

  int64_t launches() const override { return nl; }
  void use_graphs(bool on) override { graphs = on; }

  bool init(pic_ctx* const* runs, int nr, cudaStream_t st, std::string* why) {
    n = nr;
    s = st;
    if (n < 1 || n > 512) { *why = "ensemble size outside 1..512"; return false; }
    const pic_config& c0 = runs[0]->cfg;
    for (int r = 0; r < n; r++) {
      pic_ctx* c = runs[r];
      if (c->s3 || !c->sim || c->stream != st) { *why = "3D, 1D or differently streamed run"; return false; }
      const pic_config& cf = c->cfg;
      if (cf.precision != c0.precision || cf.shape_order != c0.shape_order) { *why = "mixed precisions or orders"; return false; }
      Sim<T>* m = S<T>(c);
      if (!m->batchable()) { *why = "run with lab samples, moving window or node gather"; return false; }
      sims.push_back(m);
    }
    Sim<T>* m0 = sims[0];
    order = c0.shape_order;
    friedman = m0->friedman;
    ck = runs[0]->hg.b2 != 0.0;
    filt_gather = m0->filt_gather;
    filt_J = m0->filt_J;
    const FilterTaps<T> ft0 = filter_taps<T>(m0->fs);
    pt_taps = filter_taps_class<T>(ft0);
    smem_nodes = m0->smem_nodes;
    tile_z = m0->sb.tz;
    push_grid = m0->push_grid;
    filt_smem = tile_smem_bytes<T>(m0->tmaps, filt_gather ? ft0.H : 0);
    fused_smem = filt_gather ? faraday_fused_smem<T>(m0->tmaps, ft0.H, pt_taps, friedman) : 0;
    amp_smem = tile_smem_bytes<T>(m0->tmaps, filt_J ? ft0.H : 0);
    std::vector<int> tile_off(n + 1), ion_off(n + 1), inj_off(n + 1), ant_off(n + 1);
    for (int r = 0; r < n; r++) {
      Sim<T>* m = sims[r];
      const bool ck_r = runs[r]->hg.b2 != 0.0;
      const FilterTaps<T> ft = filter_taps<T>(m->fs);
      if (m->friedman != friedman || ck_r != ck || m->filt_gather != filt_gather || m->filt_J != filt_J ||
          filter_taps_class<T>(ft) != pt_taps || ft.H != ft0.H || m->smem_nodes != smem_nodes ||
          m->sb.tz != tile_z || m->tmaps.H != m0->tmaps.H) {
        *why = "runs differ in solver family, damping, filter or particle tile";
        return false;
      }
      if (fused_smem > 0 && faraday_fused_smem<T>(m->tmaps, ft.H, pt_taps, friedman) == 0) fused_smem = 0;
      int tk, ti;
      field_tiles(m->g, tk, ti);
      tile_off[r + 1] = tile_off[r] + tk * ti;
      const bool column = m->ions && !m->pairs;
      any_ion = any_ion || column;
      ion_off[r + 1] = ion_off[r] + (column ? (int)((m->ion_rows_max() + 255) / 256) : 0);
      inj_off[r + 1] = inj_off[r] + m->inj_xblocks() * m->inj_rblocks_max();
      ant_off[r + 1] = ant_off[r] + (std::max(m->g.nx, m->g.nz) + 1 + 127) / 128;
      beam_blocks = std::max(beam_blocks, (m->beam.n + 127) / 128);
    }
    bg.nruns = n;
    bg.tiles = tile_off[n];
    bg.ion_blocks = ion_off[n];
    bg.inj_blocks = inj_off[n];
    bg.ant_blocks = ant_off[n];
    pic_ctx* c0x = runs[0];
    int* off = (int*)c0x->dalloc(sizeof(int) * 4 * (n + 1) + 64);
    bg.push_counter = (int*)c0x->dalloc(sizeof(int));
    for (int q = 0; q < 2; q++) dA[q] = (StepArgs<T>*)c0x->dalloc(sizeof(StepArgs<T>) * n);
    if (!off || !bg.push_counter || !dA[0] || !dA[1]) { *why = "batch allocation failed"; return false; }
    std::vector<int> all;
    for (auto* v : {&tile_off, &ion_off, &inj_off, &ant_off}) all.insert(all.end(), v->begin(), v->end());
    cudaMemcpyAsync(off, all.data(), sizeof(int) * all.size(), cudaMemcpyHostToDevice, s);
    bg.tile_off = off;
    bg.ion_off = off + (n + 1);
    bg.inj_off = off + 2 * (n + 1);
    bg.ant_off = off + 3 * (n + 1);
    for (int q = 0; q < 2; q++) {
      if (cudaMallocHost(&hA[q], sizeof(StepArgs<T>) * n) != cudaSuccess ||
          cudaEventCreateWithFlags(&done[q], cudaEventDisableTiming) != cudaSuccess) {
        *why = "pinned buffer or event creation failed";
        return false;
      }
      std::memset(static_cast<void*>(hA[q]), 0, sizeof(StepArgs<T>) * n);
    }
    cudaStreamSynchronize(s);
    return cudaGetLastError() == cudaSuccess;
  }

  void enqueue(int q) {
    cudaMemcpyAsync(dA[q], hA[q], sizeof(StepArgs<T>) * n, cudaMemcpyHostToDevice, s);
    launch_faraday_filter_batch<T>(dA[q], bg, friedman, ck, pt_taps, filt_gather, filt_smem, fused_smem, s);
    launch_push_batch<T>(dA[q], bg, order, push_grid, smem_nodes, tile_z, s);
    launch_beam_push_batch<T>(dA[q], n, beam_blocks, s);
    launch_antenna_ion_batch<T>(dA[q], bg, any_ion, s);
    launch_ampere_batch<T>(dA[q], bg, filt_J, pt_taps, amp_smem, s);
    launch_inject_batch<T>(dA[q], bg, s);
  }
  static int kernels_per_step(bool filt, bool ion, bool beam) {
    return 1 + (filt ? 1 : 0) + 3 + (beam ? 1 : 0) + 1 + (ion ? 1 : 0) + 1 + 2;
  }

  int step(int nsteps) override {
    for (int k = 0; k < nsteps; k++) {
      const int q = (int)(nstep & 1);
      // the slot's previous use (its host-to-device copy) must be over before its host buffer is refilled
      if (used[q]) cudaEventSynchronize(done[q]);
      std::vector<int> sorts;
      for (int r = 0; r < n; r++) {
        bool srt = false;
        if (!sims[r]->batchable()) return sims[r]->c->fail(PIC_ESTATE, "batched ensemble: a run gained lab samples");
        const int rc = sims[r]->plan_step(hA[q][r], srt);
        if (rc != PIC_OK) return rc;
        if (srt) sorts.push_back(r);
      }
      if (graphs) {
        if (!gx[q]) {
          if (nstep < 2) {
            // the first step of each slot runs uncaptured (function attributes set, modules loaded)
            enqueue(q);
          } else {
            cudaGraph_t gr = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) return PIC_ECUDA;
            enqueue(q);
            if (cudaStreamEndCapture(s, &gr) != cudaSuccess || !gr) return PIC_ECUDA;
            const cudaError_t e = cudaGraphInstantiate(&gx[q], gr, 0);
            cudaGraphDestroy(gr);
            if (e != cudaSuccess) return PIC_ECUDA;
          }
        }
        if (gx[q] && cudaGraphLaunch(gx[q], s) != cudaSuccess) return PIC_ECUDA;
      } else {
        enqueue(q);
      }
      cudaEventRecord(done[q], s);
      used[q] = true;
      nl += kernels_per_step(filt_gather, any_ion, beam_blocks > 0);
      for (int r : sorts) {
        sims[r]->do_sort();
        nl += 8;
      }
      nstep++;
    }
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
  }
};

}  // namespace

Batch* picgb::make_batch(pic_ctx* const* runs, int n, cudaStream_t s, std::string* why) {
  if (n < 1 || !runs[0]->sim) {
    *why = "no 2D runs";
    return nullptr;
  }
  Batch* b = nullptr;
  bool ok = false;
  if (runs[0]->cfg.precision == PIC_FP64) {
    auto* x = new BatchImpl<double>();
    ok = x->init(runs, n, s, why);
    b = x;
  } else {
    auto* x = new BatchImpl<float>();
    ok = x->init(runs, n, s, why);
    b = x;
  }
  if (!ok) {
    delete b;
    return nullptr;
  }
  return b;
}


extern "C" {

int pic_init(const pic_config* cfg, pic_alloc_fn alloc, pic_free_fn free_fn, void* alloc_user, void* cuda_stream,
             pic_ctx** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (!cfg || cfg->struct_size != sizeof(pic_config) || cfg->version != PIC_API_VERSION) return PIC_EINVAL;
  if (cfg->dim != 1 && cfg->dim != 2 && cfg->dim != 3) return PIC_EINVAL;
  if (cfg->gather_scheme != 0 && cfg->gather_scheme != 1) return PIC_EINVAL;
  // the composed filter: at most 16 passes per stride and a halo of at most FILTER_HMAX cells; a stride set
  // is non-negative and 0-terminated
  FilterSpec fs0{};
  fs0.passes = cfg->filter_passes; fs0.stride = cfg->filter_stride; fs0.compensate = cfg->filter_compensate;
  for (int q = 0; q < 4; q++) {
    fs0.strides[q] = cfg->filter_stride_set[q];
    if (fs0.strides[q] < 0 || (q > 0 && fs0.strides[q] > 0 && fs0.strides[q - 1] <= 0)) return PIC_EINVAL;
  }
  const int Hf = filter_halo(fs0);
  if (cfg->filter_passes + (cfg->filter_compensate ? 1 : 0) > 16 || Hf > FILTER_HMAX) return PIC_EINVAL;
  if (cfg->dim == 1) {
    if (cfg->nz < 16 || !(cfg->dz_lab > 0)) return PIC_EINVAL;
    if (cfg->shape_order != 1 && cfg->shape_order != 3) return PIC_EINVAL;
    if (cfg->precision != PIC_FP64 && cfg->precision != PIC_MIXED) return PIC_EINVAL;
    if (cfg->theta < 0 || cfg->theta > 1) return PIC_EINVAL;
    if (cfg->filter_passes < 0 || cfg->filter_stride < 1 || cfg->pml_cells < 0) return PIC_EINVAL;
    std::unique_ptr<pic_ctx> c(new pic_ctx());
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->alloc = alloc; c->freef = free_fn; c->user = alloc_user;
    int st = PIC_OK;
    std::string e;
    c->s3.reset(picgb::make_sim1(cfg, alloc, free_fn, alloc_user, c->stream, &st, &e));
    if (!c->s3) return st;
    *out = c.release();
    return PIC_OK;
  }
  if (cfg->dim == 3) {
    if (cfg->nx < 8 || cfg->nz < 8 || !(cfg->dx > 0) || !(cfg->dz_lab > 0)) return PIC_EINVAL;
    if (cfg->shape_order != 1 && cfg->shape_order != 3) return PIC_EINVAL;
    if (cfg->precision != PIC_FP64 && cfg->precision != PIC_MIXED) return PIC_EINVAL;
    if (std::fabs(cfg->ck_alpha + 4 * cfg->ck_beta + 4 * cfg->ck_gamma - 1.0) > 1e-12) return PIC_EINVAL;
    if (cfg->theta < 0 || cfg->theta > 1) return PIC_EINVAL;
    if (cfg->filter_passes < 0 || cfg->filter_stride < 1 || cfg->pml_cells < 0) return PIC_EINVAL;
    std::unique_ptr<pic_ctx> c(new pic_ctx());
    c->cfg = *cfg;
    c->stream = (cudaStream_t)cuda_stream;
    c->alloc = alloc; c->freef = free_fn; c->user = alloc_user;
    int st = PIC_OK;
    std::string e;
    c->s3.reset(picgb::make_sim3(cfg, alloc, free_fn, alloc_user, c->stream, &st, &e));
    if (!c->s3) return st;
    *out = c.release();
    return PIC_OK;
  }
  if (cfg->nx < 8 || cfg->nz < 8 || !(cfg->dx > 0) || !(cfg->dz_lab > 0)) return PIC_EINVAL;
  if (cfg->shape_order != 1 && cfg->shape_order != 3) return PIC_EINVAL;
  if (cfg->precision != PIC_FP64 && cfg->precision != PIC_MIXED) return PIC_EINVAL;
  if (std::fabs(cfg->ck_alpha + 4 * cfg->ck_beta + 4 * cfg->ck_gamma - 1.0) > 1e-12) return PIC_EINVAL;
  if (cfg->theta < 0 || cfg->theta > 1) return PIC_EINVAL;
  if (cfg->filter_passes < 0 || cfg->filter_stride < 1 || cfg->pml_cells < 0) return PIC_EINVAL;
  std::unique_ptr<pic_ctx> c(new pic_ctx());
  c->cfg = *cfg;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = alloc; c->freef = free_fn; c->user = alloc_user;
  HostGeom& h = c->hg;
  h.gamma = cfg->gamma_boost < 1.0 ? 1.0 : cfg->gamma_boost;
  h.beta = std::sqrt(1.0 - 1.0 / (h.gamma * h.gamma));
  h.dz = (1.0 + h.beta) * h.gamma * cfg->dz_lab;     // Sec. 5.1.1
  h.dx = cfg->dx;
  h.a2 = cfg->ck_alpha + 2.0 * cfg->ck_beta;         // PR-3
  h.b2 = cfg->ck_beta + 2.0 * cfg->ck_gamma;
  h.dt_cfl = cfl_2d(cfg->ck_alpha, cfg->ck_gamma, h.dx, h.dz, cfg->theta);
  h.dt = cfg->dt > 0.0 ? cfg->dt : cfg->courant * h.dt_cfl;
  if (!(h.dt > 0.0)) return PIC_EINVAL;
  if (h.dt > h.dt_cfl * (1.0 + 1e-12)) return PIC_ECFL;
  h.guard = cfg->particle_guard >= 0 ? cfg->particle_guard : (cfg->shape_order == 3 ? 3 : 2) + Hf + 2;
  // particles must not read filtered fields, nor deposit current, within reach of the walls (PR-10)
  if (h.guard < (cfg->shape_order == 3 ? 3 : 2) + Hf + 1) return PIC_EINVAL;
  const int L = cfg->pml_cells;
  h.gx_lo = L + h.guard; h.gx_hi = cfg->nx - L - h.guard;
  h.gz_lo = L + h.guard; h.gz_hi = cfg->nz - L - h.guard;
  if (h.gx_hi - h.gx_lo < 2 || h.gz_hi - h.gz_lo < 2) return PIC_EINVAL;
  if (h.gx_lo < 4 || h.gz_lo < 4) return PIC_EINVAL;
  const int elem = cfg->precision == PIC_FP64 ? 8 : 4;
  const int align = 128 / elem;
  h.ld = ((cfg->nz + 1 + align - 1) / align) * align;
  int r;
  if (cfg->precision == PIC_FP64) {
    auto* s = new Sim<double>(c.get());
    c->sim.reset(s);
    r = s->init();
  } else {
    auto* s = new Sim<float>(c.get());
    c->sim.reset(s);
    r = s->init();
  }
  if (r != PIC_OK) {
    c->sim.reset();
    c->release_all();
    return r;
  }
  cudaStreamSynchronize(c->stream);
  *out = c.release();
  return PIC_OK;
}

int pic_load_plasma(pic_ctx* c, const pic_plasma* p) {
  if (!c) return PIC_EINVAL;
  if (!p || p->struct_size != sizeof(pic_plasma) || p->version != PIC_API_VERSION) return c->fail(PIC_EINVAL, "bad pic_plasma");
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->load_plasma(p);
  return DISPATCH(c, load_plasma(p));
}

int pic_inject_laser(pic_ctx* c, const pic_laser* l) {
  if (!c) return PIC_EINVAL;
  if (!l || l->struct_size != sizeof(pic_laser) || l->version != PIC_API_VERSION) return c->fail(PIC_EINVAL, "bad pic_laser");
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->set_laser(l);
  return DISPATCH(c, set_laser(l));
}

int pic_step(pic_ctx* c, int nsteps) {
  if (!c) return PIC_EINVAL;
  if (nsteps < 0) return c->fail(PIC_EINVAL, "nsteps < 0");
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->run(nsteps);
  return DISPATCH(c, run(nsteps));
}

int pic_sync(pic_ctx* c) {
  if (!c) return PIC_EINVAL;
  if (c->s3) return c->s3->sync();
  int r = DISPATCH(c, sync());
  return c->status != PIC_OK ? c->status : r;
}

int pic_boosted_to_lab_diag(pic_ctx* c, const pic_btd_req* req, pic_btd_out* out) {
  if (!c) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (req && !out) {
    if (req->struct_size != sizeof(pic_btd_req) || req->version != PIC_API_VERSION) return c->fail(PIC_EINVAL, "bad pic_btd_req");
    if (c->s3) return c->s3->btd_set(req);
    return DISPATCH(c, btd_set(req));
  }
  if (!req && out) {
    if (out->struct_size != sizeof(pic_btd_out) || out->version != PIC_API_VERSION) return c->fail(PIC_EINVAL, "bad pic_btd_out");
    if (c->s3) return c->s3->btd_get(out);
    return DISPATCH(c, btd_get(out));
  }
  return c->fail(PIC_EINVAL, "pass exactly one of req and out");
}

int pic_free(pic_ctx* c) {
  if (!c) return PIC_OK;
  cudaStreamSynchronize(c->stream);
  c->s3.reset();
  c->sim.reset();
  c->release_all();
  delete c;
  return PIC_OK;
}

int pic_get_field(pic_ctx* c, int comp, double* dst, int on_device) {
  if (!c || !dst) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->get_field(comp, dst, on_device);
  return DISPATCH(c, get_field(comp, dst, on_device));
}

int pic_get_rho_noalloc(pic_ctx* c, double* dst_device) {
  if (!c || !dst_device) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->fail(PIC_EINVAL, "pic_get_rho_noalloc: 2D contexts only");
  if (c->cfg.nz > PIC_NOALLOC_MAX_NZ) return c->fail(PIC_EINVAL, "pic_get_rho_noalloc: nz exceeds PIC_NOALLOC_MAX_NZ");
  return DISPATCH(c, get_rho_noalloc(dst_device));
}

int pic_beam_self_field(pic_ctx* c) {
  if (!c) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (c->s3) {
    const int r = c->s3->beam_self_field();
    if (r != PIC_OK) return c->fail(r, c->s3->error().empty() ? "pic_beam_self_field: 1D contexts have no test beam"
                                                              : c->s3->error());
    return PIC_OK;
  }
  return DISPATCH(c, beam_self_field());
}

int pic_set_field(pic_ctx* c, int comp, const double* src) {
  if (!c || !src) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->set_field(comp, src);
  return DISPATCH(c, set_field(comp, src));
}

int pic_get_particles(pic_ctx* c, int species, double* x, double* z, double* ux, double* uy, double* uz, double* w,
                      uint32_t* id, int32_t* flags, int64_t* count) {
  if (!c || !count) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->get_particles(species, x, nullptr, z, ux, uy, uz, w, id, flags, count);
  return DISPATCH(c, get_particles(species, x, z, ux, uy, uz, w, id, flags, count));
}

int pic_get_particles_y(pic_ctx* c, int species, double* y, int64_t* count) {
  if (!c || !count) return PIC_EINVAL;
  if (c->status != PIC_OK) return c->status;
  if (!c->s3) return c->fail(PIC_EINVAL, "pic_get_particles_y: 3D contexts only");
  if (!y) return c->s3->get_particles(species, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr,
                                      nullptr, count);
  return c->s3->get_particles(species, nullptr, y, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, count);
}

int pic_get_stats(pic_ctx* c, pic_stats* out) {
  if (!c || !out) return PIC_EINVAL;
  if (out->struct_size != sizeof(pic_stats) || out->version != PIC_API_VERSION) return c->fail(PIC_EINVAL, "bad pic_stats");
  if (c->status != PIC_OK) return c->status;
  if (c->s3) return c->s3->stats(out);
  return DISPATCH(c, stats(out));
}

const char* pic_last_error(pic_ctx* c) {
  if (!c) return "null context";
  if (c->s3) return c->s3->error().c_str();
  return c->err.empty() ? "" : c->err.c_str();
}

int64_t pic_kernel_launches(pic_ctx* c) {
  if (!c) return 0;
  return c->s3 ? c->s3->launches() : c->launches;
}

int pic_kernel_timing(pic_ctx* c, int enable, int which, double* ms_total, int64_t* launches) {
  if (!c) return PIC_EINVAL;
  if (c->s3) return c->s3->kernel_timing(enable, which, ms_total, launches);
  return DISPATCH(c, kernel_timing(enable, which, ms_total, launches));
}

}  // extern "C"
