// Particle kernels of the boosted-frame PIC step:
//  - k_push: persistent gather -> Boris -> move -> Esirkepov kernel. One CTA
//    takes one chunk (a contiguous run of particles whose cells lie in a known
//    bounding box), stages the six gather fields of the box in shared memory,
//    deposits J into a shared-memory copy of the box with shared atomics and
//    adds the box to the global current once. A chunk whose box exceeds the
//    shared-memory capacity runs the same arithmetic on global memory.
//  - tile sort (counting sort into tiles; within a tile, particles are grouped
//    by their rank inside their cell so that the lanes of a warp usually hold
//    particles of different cells and their shared atomics do not collide);
//  - plasma rows entering through the +z plane (Sec. 3.1.1, PR-12).
#include <climits>
#include <cstring>
#include <type_traits>

#include "pic_common.cuh"

namespace picgb {

namespace {

constexpr int PB_THREADS = 256;

template <int ORDER>
struct St;
template <>
struct St<3> { static constexpr int NG = 4, ND = 5, LO = 2, HI = 3; };
template <>
struct St<1> { static constexpr int NG = 2, ND = 3, LO = 1, HI = 2; };

template <class T, int ORDER>
__device__ __forceinline__ void wts(T t, T* w) {
  if (ORDER == 3) weights3<T>(t, w);
  else weights1<T>(t, w);
}

// place NG weights of a particle whose first node is at offset o (0 or 1) into an ND window
template <class T, int ORDER>
__device__ __forceinline__ void place(const T* w, int o, T* S) {
  constexpr int NG = St<ORDER>::NG, ND = St<ORDER>::ND;
#pragma unroll
  for (int j = 0; j < ND; j++) {
    T a = (j < NG) ? w[j] : T(0);
    T b = (j >= 1) ? w[j - 1] : T(0);
    S[j] = o ? b : a;
  }
}

// interpolation of one component from a block addressed as (i - ox)*ld + (k - oz)
template <class T, int ORDER>
__device__ __forceinline__ T interp(const T* F, int ld, int ox, int oz, int fi, int fk, const T* wx, const T* wz) {
  constexpr int NG = St<ORDER>::NG;
  const int off = ORDER == 3 ? 1 : 0;
  T acc = T(0);
  const T* row = F + (long)(fi - off - ox) * ld + (fk - off - oz);
#pragma unroll
  for (int a = 0; a < NG; a++) {
    T r = T(0);
#pragma unroll
    for (int b = 0; b < NG; b++) r += row[b] * wz[b];
    acc += r * wx[a];
    row += ld;
  }
  return acc;
}

template <class T>
struct Vec2;
template <>
struct Vec2<float> { typedef float2 type; };
template <>
struct Vec2<double> { typedef double2 type; };

// interpolation of two components stored as pairs at the same Yee location
template <class T, int ORDER>
__device__ __forceinline__ void interp2(const typename Vec2<T>::type* F, int ld, int ox, int oz, int fi, int fk,
                                        const T* wx, const T* wz, T& r0, T& r1) {
  constexpr int NG = St<ORDER>::NG;
  const int off = ORDER == 3 ? 1 : 0;
  T a0 = T(0), a1 = T(0);
  const typename Vec2<T>::type* row = F + (fi - off - ox) * ld + (fk - off - oz);
#pragma unroll
  for (int a = 0; a < NG; a++) {
    T s0 = T(0), s1 = T(0);
#pragma unroll
    for (int b = 0; b < NG; b++) {
      const typename Vec2<T>::type v = row[b];
      s0 += v.x * wz[b];
      s1 += v.y * wz[b];
    }
    a0 += s0 * wx[a];
    a1 += s1 * wx[a];
    row += ld;
  }
  r0 = a0;
  r1 = a1;
}


// products and differences rounded on their own (no contraction into FMA)
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Lab-fixed ion of a lattice site (mixed path): its stored cell and offsets,
// grid cells at t^n and t^{n+1}, and the shape weights of its Esirkepov J_z on
// the window starting at (bx, bz) (bx, bz are set when set_window).
template <int ORDER>
struct IonSite {
  uint32_t cell;
  float ox, oz;
  int fx, fz0, fz1;
  float tz0, tz1;
};

__device__ __forceinline__ int site_row(uint32_t id, const PushConst& pc) { return (int)(id >> pc.kb); }

template <int ORDER>
__device__ __forceinline__ void ion_site(uint32_t id, const PushConst& pc, IonSite<ORDER>& s) {
  lattice_site_pow2(id, pc.kb, pc.lpx, pc.lpz, pc.gx_lo, pc.z0_cells, s.cell, s.ox, s.oz);
  s.fx = cell_x(s.cell);
  frame_z(s.cell, s.oz, pc.fr0_sz, pc.fr0_fz, s.fz0, s.tz0);
  frame_z(s.cell, s.oz, pc.fr1_sz, pc.fr1_fz, s.fz1, s.tz1);
}

// Esirkepov current of one particle on an NDX (x) by ND (z) window whose first
// node is Jx (Jy, Jz follow at component stride cs). The weights factorise:
// Jx(a,b) = Px[a] Fz[b] with Px the running sum of cx DSx and Fz = S0z + DSz/2
// (likewise Jz), and Wy = S0z (S0x + DSx/2) + DSz (S0x/2 + DSx/3). Zero
// contributions are skipped (a slot that is zero on every lane of a warp costs
// no shared-memory wavefront).
//
// JZ: 0 = no J_z, 1 = the particle's J_z, 2 = the particle's J_z minus that of a
// particle with x weights Sxi and z weight change DSzi on the same window (the
// electron and its lattice ion): the two are combined before the atomic, with
// separately rounded products, so that the large streaming currents cancel in
// registers instead of in the accumulated current.
template <class T, int ND, int NDX, bool SMEM>
__device__ __forceinline__ void deposit(T* Jx, long cs, int ld, const T* S0x, const T* DSx, const T* S0z, const T* DSz,
                                        T cx, T cy, T cz, int JZ = 1, const T* Sxi = nullptr,
                                        const T* DSzi = nullptr) {
  typedef typename std::conditional<SMEM, int, long>::type Idx;
  T* Jy = Jx + cs;
  T* Jz = Jx + 2 * cs;
  // J_x, then J_y, then J_z: each axis's running sums are formed where they are used
  {
    T Px[NDX - 1];
    T ax = T(0);
#pragma unroll
    for (int a = 0; a < NDX - 1; a++) { ax += cx * DSx[a]; Px[a] = ax; }
#pragma unroll
    for (int b = 0; b < ND; b++) {
      const T fzb = S0z[b] + T(0.5) * DSz[b];
#pragma unroll
      for (int a = 0; a < NDX - 1; a++) {
        const T v = Px[a] * fzb;
        if (v != T(0)) atomicAdd(Jx + (Idx)a * ld + b, v);
      }
    }
  }
  if (cy != T(0)) {
#pragma unroll
    for (int a = 0; a < NDX; a++) {
      const T ay = cy * (S0x[a] + T(0.5) * DSx[a]);
      const T by = cy * (T(0.5) * S0x[a] + DSx[a] * T(1.0 / 3.0));
#pragma unroll
      for (int b = 0; b < ND; b++) {
        const T v = ay * S0z[b] + by * DSz[b];
        if (v != T(0)) atomicAdd(Jy + (Idx)a * ld + b, v);
      }
    }
  }
  if (JZ != 0) {
    T Pz[ND - 1], Pzi[ND - 1];
    T az = T(0), ai = T(0);
#pragma unroll
    for (int b = 0; b < ND - 1; b++) {
      az += cz * DSz[b]; Pz[b] = az;
      if (JZ == 2) { ai += cz * DSzi[b]; Pzi[b] = ai; }
    }
#pragma unroll
    for (int a = 0; a < NDX; a++) {
      const T fxa = S0x[a] + T(0.5) * DSx[a];
#pragma unroll
      for (int b = 0; b < ND - 1; b++) {
        T v;
        if (JZ == 2) v = sub_rn(mul_rn(fxa, Pz[b]), mul_rn(Sxi[a], Pzi[b]));
        else v = fxa * Pz[b];
        if (v != T(0)) atomicAdd(Jz + (Idx)a * ld + b, v);
      }
    }
  }
}

// J_z of a lab-fixed ion alone (its electron has left, or their windows
// differ): the electron formula with the same weight and the opposite charge
template <class T, int ORDER, bool SMEM>
__device__ __forceinline__ void ion_jz(T* Jb, long cs, int ld, int ox, int oz, const IonSite<ORDER>& s, T cz) {
  constexpr int NG = St<ORDER>::NG, ND = St<ORDER>::ND;
  typedef typename std::conditional<SMEM, int, long>::type Idx;
  const int off = ORDER == 3 ? 1 : 0;
  T wx[NG], w0[NG], w1[NG];
  wts<T, ORDER>(T(s.ox), wx);
  wts<T, ORDER>(T(s.tz0), w0);
  wts<T, ORDER>(T(s.tz1), w1);
  const int bx = s.fx - off, bz = min(s.fz0, s.fz1) - off;
  T S0z[ND], S1z[ND];
  place<T, ORDER>(w0, s.fz0 - off - bz, S0z);
  place<T, ORDER>(w1, s.fz1 - off - bz, S1z);
  T* Jz = Jb + 2 * cs + (Idx)(bx - ox) * ld + (bz - oz);
  T Pz[ND - 1];
  T az = T(0);
#pragma unroll
  for (int b = 0; b < ND - 1; b++) { az += cz * (S1z[b] - S0z[b]); Pz[b] = az; }
#pragma unroll
  for (int a = 0; a < NG; a++) {
#pragma unroll
    for (int b = 0; b < ND - 1; b++) {
      const T v = -(wx[a] * Pz[b]);
      if (v != T(0)) atomicAdd(Jz + (Idx)a * ld + b, v);
    }
  }
}

// Cells of the chunk's box (inclusive): a particle whose cell at t^n, or whose
// lab-fixed ion's cell, lies outside it is not in the staged window.
struct Box {
  int ix0, ix1, iz0, iz1;
  __device__ __forceinline__ bool in(int fx, int fz) const { return fx >= ix0 && fx <= ix1 && fz >= iz0 && fz <= iz1; }
};

// mixed path, cubic or linear shapes: the gather of two components stored as a
// pair at one Yee location (weights wx, wz shared) with packed FP32 FMAs, and
// of two components at different locations (separate windows and weights),
// also packed: each lane of the pair rounds exactly like the scalar FMA
template <int ORDER>
__device__ __forceinline__ float2 interp_pair_f(const float2* __restrict__ F, int base, int ld, const float* wx,
                                               const float* wz) {
  constexpr int NG = St<ORDER>::NG;
  float2 acc = make_float2(0.0f, 0.0f);
  const float2* row = F + base;
#pragma unroll
  for (int a = 0; a < NG; a++) {
    float2 sacc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < NG; b++) sacc = __ffma2_rn(row[b], make_float2(wz[b], wz[b]), sacc);
    acc = __ffma2_rn(sacc, make_float2(wx[a], wx[a]), acc);
    row += ld;
  }
  return acc;
}
template <int ORDER>
__device__ __forceinline__ float2 interp_two_f(const float* __restrict__ F0, int base0, const float* __restrict__ F1,
                                              int base1, int ld, const float* wx0, const float* wz0,
                                              const float* wx1, const float* wz1) {
  constexpr int NG = St<ORDER>::NG;
  float2 acc = make_float2(0.0f, 0.0f);
  const float* r0 = F0 + base0;
  const float* r1 = F1 + base1;
#pragma unroll
  for (int a = 0; a < NG; a++) {
    float2 sacc = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int b = 0; b < NG; b++) sacc = __ffma2_rn(make_float2(r0[b], r1[b]), make_float2(wz0[b], wz1[b]), sacc);
    acc = __ffma2_rn(sacc, make_float2(wx0[a], wx1[a]), acc);
    r0 += ld;
    r1 += ld;
  }
  return acc;
}

// Mixed path: the state of a thread's next particle is copied into shared memory by per-thread
// asynchronous copies while the thread pushes the current one (each thread reads only what it copied
// itself: no block barrier). Word k of a thread's record sits at rec[k * PB_THREADS] (a warp's reads fall
// in consecutive banks); the record is read into registers before the next copy overwrites it.
enum { RW_W, RW_CELL, RW_OX, RW_OZ, RW_UX, RW_UY, RW_UZ, RW_ID, RW_N };
struct PRec { uint32_t v[RW_N]; };

template <class T>
constexpr size_t push_stage_bytes() { return CellPos<T>::value ? (size_t)RW_N * PB_THREADS * 4 : 0; }

__device__ __forceinline__ void cp_async4(uint32_t* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void stage_particle(const Particles<float>& p, int pi, uint32_t* rec) {
  cp_async4(rec + RW_W * PB_THREADS, p.w + pi);
  cp_async4(rec + RW_CELL * PB_THREADS, p.cell + pi);
  cp_async4(rec + RW_OX * PB_THREADS, p.ox + pi);
  cp_async4(rec + RW_OZ * PB_THREADS, p.oz + pi);
  cp_async4(rec + RW_UX * PB_THREADS, p.ux + pi);
  cp_async4(rec + RW_UY * PB_THREADS, p.uy + pi);
  cp_async4(rec + RW_UZ * PB_THREADS, p.uz + pi);
  cp_async4(rec + RW_ID * PB_THREADS, p.id + pi);
}

// a particle's word from its record (ST) or from global memory
template <bool ST, class X>
__device__ __forceinline__ X pword(const X* g, int pi, const PRec* r, int k) {
  if constexpr (ST) {
    static_assert(sizeof(X) == 4, "records hold 32-bit words");
    X x;
    memcpy(&x, &r->v[k], 4);
    return x;
  } else {
    return g[pi];
  }
}

// Bounding box of the cells a thread's particles occupy, accumulated over its particles of a chunk.
struct BoxI {
  int x0 = INT_MAX, x1 = INT_MIN, z0 = INT_MAX, z1 = INT_MIN;
  __device__ __forceinline__ void add(int x, int z) {
    x0 = min(x0, x); x1 = max(x1, x); z0 = min(z0, z); z1 = max(z1, z);
  }
  __device__ __forceinline__ BoxI unpack() const { return *this; }
};
// The same in two registers, (x, z) as unsigned 16-bit halves: mixed-path cells are 16-bit and the
// window path only adds cells of its own non-negative window
struct BoxP {
  uint32_t lo = 0xffffffffu, hi = 0u;
  __device__ __forceinline__ void add(int x, int z) {
    const uint32_t v = ((uint32_t)x << 16) | ((uint32_t)z & 0xffffu);
    lo = __vminu2(lo, v); hi = __vmaxu2(hi, v);
  }
  __device__ __forceinline__ BoxI unpack() const {
    BoxI b;
    if ((lo >> 16) <= (hi >> 16)) {   // something was added
      b.x0 = (int)(lo >> 16); b.x1 = (int)(hi >> 16); b.z0 = (int)(lo & 0xffffu); b.z1 = (int)(hi & 0xffffu);
    }
    return b;
  }
};

// One particle: gather -> Boris -> move -> Esirkepov. E/B/J are 3-component
// blocks (component stride cs) addressed as (i - ox)*ld + (k - oz). With SMEM
// the fields are the shared-memory window: pairs (Ex, Bz) and (Ez, Bx), which
// share a Yee location, then Ey and By, each block cs elements long (Bb unused).
// With SMEM the particle must lie in the staged window: when its cell at t^n
// (or its live lattice ion's cell) is outside the chunk's box, nothing is
// changed and false is returned, so that the caller takes the global path.
// The cells of the particle's new position (and of its ion) are added to acc; with ST the particle's
// state comes from its record rec instead of the arrays of p.
template <class T, int ORDER, bool SMEM, bool MC = false, class ACC = BoxI, bool ST = false>
__device__ __forceinline__ bool push_one(const T* __restrict__ Eb, const T* __restrict__ Bb, T* Jb, long cs, int ld,
                                         int ox, int oz, const Particles<T>& p, int pi, const PushConst& pc, const Box& box,
                                         ACC& acc,
                                         const PRec* rec = nullptr) {
  constexpr int NG = St<ORDER>::NG, ND = St<ORDER>::ND;
  constexpr bool CP = CellPos<T>::value;
  const T w = pword<ST>(p.w, pi, rec, RW_W);
  if (w == T(0)) return true;
  if constexpr (CP) {
    if (w < T(0)) {
      // ghost: the lab-fixed ion of an electron that has left the domain; it
      // deposits its J_z until its lattice row leaves too
      const uint32_t id = pword<ST>(p.id, pi, rec, RW_ID);
      if (site_row(id, pc) < pc.mlo) { p.w[pi] = T(0); return true; }
      IonSite<ORDER> is;
      ion_site<ORDER>(id, pc, is);
      if (SMEM && !box.in(is.fx, is.fz0)) return false;
      ion_jz<T, ORDER, SMEM>(Jb, cs, ld, ox, oz, is, pc.kz_f * (-w));
      acc.add(is.fx, is.fz1);
      return true;
    }
  }
  int fx, fz, fxh, fzh;
  T tx, tz, txh, tzh;
  double x = 0.0, z = 0.0, X = 0.0, Z = 0.0;
  uint32_t cs0 = 0;   // mixed path: stored cell and z offset (drifting frame)
  float ozs = 0.0f;
  // the lab-fixed ion of the particle's lattice site (mixed path, electron-ion pairs)
  bool ion_live = false, at_site = false;
  uint32_t pid = 0;
  IonSite<ORDER> is{};
  if constexpr (CP) {
    cs0 = pword<ST>(p.cell, pi, rec, RW_CELL);
    ozs = pword<ST>(p.oz, pi, rec, RW_OZ);
    fx = cell_x(cs0);
    frame_z(cs0, ozs, pc.fr0_sz, pc.fr0_fz, fz, tz);
    tx = pword<ST>(p.ox, pi, rec, RW_OX);
    if (pc.pairs) {
      pid = pword<ST>(p.id, pi, rec, RW_ID);
      ion_live = site_row(pid, pc) >= pc.mlo;
      if (ion_live) {
        lattice_site_pow2(pid, pc.kb, pc.lpx, pc.lpz, pc.gx_lo, pc.z0_cells, is.cell, is.ox, is.oz);
        // an electron still at its lattice site shares its ion's grid position
        at_site = cs0 == is.cell && ozs == is.oz && tx == is.ox;
        if (SMEM && !at_site) {
          frame_z(is.cell, is.oz, pc.fr0_sz, pc.fr0_fz, is.fz0, is.tz0);
          if (!box.in(cell_x(is.cell), is.fz0)) return false;
        }
      }
    }
    if (SMEM && !box.in(fx, fz)) return false;
    fxh = tx >= T(0.5) ? fx : fx - 1; txh = tx >= T(0.5) ? tx - T(0.5) : tx + T(0.5);
    fzh = tz >= T(0.5) ? fz : fz - 1; tzh = tz >= T(0.5) ? tz - T(0.5) : tz + T(0.5);
  } else {
    x = p.x[pi]; z = p.z[pi];
    X = x / pc.dx; Z = (z - pc.z0) / pc.dz;
    if (SMEM && (!(X == X) || !(Z == Z) || fabs(X) > 1e9 || fabs(Z) > 1e9)) return false;
    fx = (int)floor(X); fz = (int)floor(Z);
    if (SMEM && !box.in(fx, fz)) return false;
    tx = T(X - fx); tz = T(Z - fz);
    const double Xh = X - 0.5, Zh = Z - 0.5;
    fxh = (int)floor(Xh); fzh = (int)floor(Zh);
    txh = T(Xh - fxh); tzh = T(Zh - fzh);
  }
  T ux = pword<ST>(p.ux, pi, rec, RW_UX), uy = pword<ST>(p.uy, pi, rec, RW_UY), uz = pword<ST>(p.uz, pi, rec, RW_UZ);
  T wxi[NG], wzi[NG], wxh[NG], wzh[NG];
  wts<T, ORDER>(tx, wxi); wts<T, ORDER>(tz, wzi);
  T Ex, Ey, Ez, Bx, By, Bz;
  constexpr int goff = ORDER == 3 ? 1 : 0;
  if constexpr (MC) {
    // 'momentum conserving' gather (Sec. 5): every gather copy already holds node values
    if constexpr (SMEM) {
      typedef typename Vec2<T>::type V2;
      interp2<T, ORDER>(reinterpret_cast<const V2*>(Eb), ld, ox, oz, fx, fz, wxi, wzi, Ex, Bz);
      interp2<T, ORDER>(reinterpret_cast<const V2*>(Eb + 2 * cs), ld, ox, oz, fx, fz, wxi, wzi, Ez, Bx);
      Ey = interp<T, ORDER>(Eb + 4 * cs, ld, ox, oz, fx, fz, wxi, wzi);
      By = interp<T, ORDER>(Eb + 5 * cs, ld, ox, oz, fx, fz, wxi, wzi);
    } else {
      Ex = interp<T, ORDER>(Eb, ld, ox, oz, fx, fz, wxi, wzi);
      Ey = interp<T, ORDER>(Eb + cs, ld, ox, oz, fx, fz, wxi, wzi);
      Ez = interp<T, ORDER>(Eb + 2 * cs, ld, ox, oz, fx, fz, wxi, wzi);
      Bx = interp<T, ORDER>(Bb, ld, ox, oz, fx, fz, wxi, wzi);
      By = interp<T, ORDER>(Bb + cs, ld, ox, oz, fx, fz, wxi, wzi);
      Bz = interp<T, ORDER>(Bb + 2 * cs, ld, ox, oz, fx, fz, wxi, wzi);
    }
  } else {
  wts<T, ORDER>(txh, wxh); wts<T, ORDER>(tzh, wzh);
  // energy-conserving gather from each component's Yee location
  if constexpr (SMEM && CP) {
    const float2* V = reinterpret_cast<const float2*>(Eb);
    const int bxh = (fxh - goff - ox) * ld, bxi = (fx - goff - ox) * ld;
    const int bzi = fz - goff - oz, bzh = fzh - goff - oz;
    const float2 exbz = interp_pair_f<ORDER>(V, bxh + bzi, ld, wxh, wzi);
    const float2 ezbx = interp_pair_f<ORDER>(V + cs, bxi + bzh, ld, wxi, wzh);
    const float2 eyby = interp_two_f<ORDER>(Eb + 4 * cs, bxi + bzi, Eb + 5 * cs, bxh + bzh, ld, wxi, wzi, wxh, wzh);
    Ex = exbz.x; Bz = exbz.y; Ez = ezbx.x; Bx = ezbx.y; Ey = eyby.x; By = eyby.y;
  } else if constexpr (SMEM) {
    typedef typename Vec2<T>::type V2;
    interp2<T, ORDER>(reinterpret_cast<const V2*>(Eb), ld, ox, oz, fxh, fz, wxh, wzi, Ex, Bz);
    interp2<T, ORDER>(reinterpret_cast<const V2*>(Eb + 2 * cs), ld, ox, oz, fx, fzh, wxi, wzh, Ez, Bx);
    Ey = interp<T, ORDER>(Eb + 4 * cs, ld, ox, oz, fx, fz, wxi, wzi);
    By = interp<T, ORDER>(Eb + 5 * cs, ld, ox, oz, fxh, fzh, wxh, wzh);
  } else {
    Ex = interp<T, ORDER>(Eb, ld, ox, oz, fxh, fz, wxh, wzi);
    Ey = interp<T, ORDER>(Eb + cs, ld, ox, oz, fx, fz, wxi, wzi);
    Ez = interp<T, ORDER>(Eb + 2 * cs, ld, ox, oz, fx, fzh, wxi, wzh);
    Bx = interp<T, ORDER>(Bb, ld, ox, oz, fx, fzh, wxi, wzh);
    By = interp<T, ORDER>(Bb + cs, ld, ox, oz, fxh, fzh, wxh, wzh);
    Bz = interp<T, ORDER>(Bb + 2 * cs, ld, ox, oz, fxh, fz, wxh, wzi);
  }
  }
  // relativistic Boris push
  T k;
  if constexpr (CP) k = pc.qm_half_f; else k = T(pc.qm_half);
  const T ic2 = T(1.0 / (kC * kC));
  T vx, vy, vz;
  if constexpr (CP) {
    // FP32 path: uz holds u_z - u0 (u0 = -gamma beta c, the plasma drift
    // momentum), so the kicks and the rotation's change of u_z keep FP32
    // precision; 1/gamma from rsqrt, 2/(1+t^2) from a fast reciprocal
    const float u0 = pc.u0z_f;
    const float umx = ux + k * Ex, umy = uy + k * Ey, dm = uz + k * Ez;
    const float kig = k * rsqrtf(pc.g0sq_f + (umx * umx + umy * umy + dm * (2.0f * u0 + dm)) * ic2);
    const float tbx = kig * Bx, tby = kig * By, tbz = kig * Bz;
    const float t2 = tbx * tbx + tby * tby + tbz * tbz;
    const float sf = __fdividef(2.0f, 1.0f + t2);
    const float sbx = sf * tbx, sby = sf * tby, sbz = sf * tbz;
    const float umz = u0 + dm;
    const float upx = umx + (umy * tbz - umz * tby);
    const float upy = umy + (umz * tbx - umx * tbz);
    const float dp = dm + (umx * tby - umy * tbx);
    const float upz = u0 + dp;
    const float plx = umx + (upy * sbz - upz * sby);
    const float ply = umy + (upz * sbx - upx * sbz);
    const float dl = dm + (upx * sby - upy * sbx);
    ux = plx + k * Ex; uy = ply + k * Ey; uz = dl + k * Ez;
    // gamma^2 - gamma0^2 from the deviation; v_z - v0 (v0 = u0/gamma0, the plasma
    // drift carried by the stored frame) formed from deviations, so that it is
    // exactly zero for a particle at the drift momentum, whose stored z stays put
    const float g2d = (ux * ux + uy * uy + uz * (2.0f * u0 + uz)) * ic2;
    const float ig1 = rsqrtf(pc.g0sq_f + g2d);
    vx = ux * ig1; vy = uy * ig1;
    const float dg = __fdividef(g2d, __fdividef(1.0f, ig1) + pc.g0_f);   // gamma - gamma0
    vz = (uz - u0 * __fdividef(dg, pc.g0_f)) * ig1;
  } else {
    T umx = ux + k * Ex, umy = uy + k * Ey, umz = uz + k * Ez;
    const T gm = sqrt(T(1) + (umx * umx + umy * umy + umz * umz) * ic2);
    const T tbx = k * Bx / gm, tby = k * By / gm, tbz = k * Bz / gm;
    const T t2 = tbx * tbx + tby * tby + tbz * tbz;
    const T sf = T(2) / (T(1) + t2);
    const T sbx = sf * tbx, sby = sf * tby, sbz = sf * tbz;
    const T upx = umx + (umy * tbz - umz * tby);
    const T upy = umy + (umz * tbx - umx * tbz);
    const T upz = umz + (umx * tby - umy * tbx);
    const T plx = umx + (upy * sbz - upz * sby);
    const T ply = umy + (upz * sbx - upx * sbz);
    const T plz = umz + (upx * sby - upy * sbx);
    ux = plx + k * Ex; uy = ply + k * Ey; uz = plz + k * Ez;
    const T g1 = sqrt(T(1) + (ux * ux + uy * uy + uz * uz) * ic2);
    vx = ux / g1; vy = uy / g1; vz = uz / g1;
  }
  // move
  int fxn, fzn;
  T txn, tzn;
  double xn = 0.0, zn = 0.0;
  uint32_t csn = 0;
  float ozn = 0.0f;
  if constexpr (CP) {
    const float ax = tx + pc.dtdx * vx, az = ozs + pc.dtdz * vz;   // z in the drifting frame
    int sx = (int)floorf(ax), sz = (int)floorf(az);
    float rx = ax - (float)sx, rz = az - (float)sz;
    if (rx >= 1.0f) { rx = 0.0f; sx++; }
    if (rz >= 1.0f) { rz = 0.0f; sz++; }
    fxn = fx + sx; txn = rx;
    csn = pack_cell(fxn, (cell_z(cs0) + sz) & 0xffff);
    ozn = rz;
    frame_z(csn, ozn, pc.fr1_sz, pc.fr1_fz, fzn, tzn);
  } else {
    xn = x + pc.dt * (double)vx;
    zn = z + pc.dt * (double)vz;
    const double Xn = xn / pc.dx, Zn = (zn - pc.z0) / pc.dz;
    fxn = (int)floor(Xn); fzn = (int)floor(Zn);
    txn = T(Xn - fxn); tzn = T(Zn - fzn);
  }
  // the lab-fixed ion of the particle's lattice site (mixed path): J_z of the
  // pair is exactly zero when electron and ion made the same move (the cold
  // streaming plasma); otherwise combined on a common window, or separate
  const int off = ORDER == 3 ? 1 : 0;
  const int bx = min(fx, fxn) - off, bz = min(fz, fzn) - off;
  int jz = 1;
  bool ion_sep = false;
  if constexpr (CP) {
    if (ion_live) {
      if (at_site && csn == cs0 && ozn == ozs && txn == tx) {
        // the pair made the same move: the ion is where the electron is
        jz = 0;
        is.fx = fxn;
        is.fz1 = fzn;
      } else {
        ion_site<ORDER>(pid, pc, is);
        if (is.fx - off == bx && min(is.fz0, is.fz1) - off == bz) jz = 2;
        else ion_sep = true;
      }
    }
  }
  T cx, cz, cy;
  if constexpr (CP) {
    cx = pc.kx_f * w; cz = pc.kz_f * w; cy = pc.ky_f * w * vy;
  } else {
    cx = T(pc.kx) * w; cz = T(pc.kz) * w; cy = T(pc.ky) * w * vy;
  }
  // the new state is stored before the deposit, which reads only registers and
  // the current window (fewer values live across it)
  bool gone;
  if constexpr (CP) {
    p.cell[pi] = csn; p.ox[pi] = txn; p.oz[pi] = ozn;
    gone = fxn < pc.cx_lo || fxn >= pc.cx_hi || fzn < pc.cz_lo || fzn >= pc.cz_hi;
  } else {
    p.x[pi] = xn; p.z[pi] = zn;
    gone = xn < pc.xlo || xn >= pc.xhi || zn < pc.zlo || zn >= pc.zhi;
  }
  p.ux[pi] = ux; p.uy[pi] = uy; p.uz[pi] = uz;
  if (gone) {
    // an electron whose ion is still inside leaves a ghost that carries the ion
    p.w[pi] = ion_live ? -w : T(0);
  } else {
    acc.add(fxn, fzn);
  }
  if constexpr (CP) {
    // the pair's ion (or the ghost's) deposits next step: its cell belongs in the chunk's box too
    if (ion_live) {
      acc.add(is.fx, is.fz1);
    }
  }
  // Esirkepov deposition on an ND x ND window. No current at all: the x weights
  // are unchanged (J_x = 0), no out-of-plane velocity (J_y = 0) and J_z cancels
  // within the pair; a warp whose lanes all carry no current skips the weights
  // and the deposit
  bool dep = !(jz == 0 && fxn == fx && txn == tx && cy == T(0));
  if constexpr (SMEM) dep = __any_sync(__activemask(), dep);
  if (dep) {
    T S0x[ND], DSx[ND], S0z[ND], DSz[ND];
    {
      // the t^n weights again (cheaper than keeping the gather's live through the push)
      T w1[NG], S1[ND];
      wts<T, ORDER>(tx, w1); place<T, ORDER>(w1, fx - off - bx, S0x);
      wts<T, ORDER>(txn, w1); place<T, ORDER>(w1, fxn - off - bx, S1);
#pragma unroll
      for (int a = 0; a < ND; a++) DSx[a] = S1[a] - S0x[a];
      wts<T, ORDER>(tz, w1); place<T, ORDER>(w1, fz - off - bz, S0z);
      wts<T, ORDER>(tzn, w1); place<T, ORDER>(w1, fzn - off - bz, S1);
#pragma unroll
      for (int a = 0; a < ND; a++) DSz[a] = S1[a] - S0z[a];
    }
    T Sxi[ND], DSzi[ND];
    if constexpr (CP) {
      if (jz == 2) {
        T wi[NG], S0i[ND], S1i[ND];
        wts<T, ORDER>(T(is.ox), wi);
        place<T, ORDER>(wi, 0, Sxi);
        wts<T, ORDER>(T(is.tz0), wi);
        place<T, ORDER>(wi, is.fz0 - off - bz, S0i);
        wts<T, ORDER>(T(is.tz1), wi);
        place<T, ORDER>(wi, is.fz1 - off - bz, S1i);
#pragma unroll
        for (int b = 0; b < ND; b++) DSzi[b] = S1i[b] - S0i[b];
      }
    }
    T* Jx = Jb + (long)(bx - ox) * ld + (bz - oz);
    if constexpr (SMEM) {
      // when no lane of the warp changes x-cell, column ND-1 of the x window is
      // empty: the warp deposits on ND-1 columns
      const bool xcross = fxn != fx;
      if (__any_sync(__activemask(), xcross))
        deposit<T, ND, ND, true>(Jx, cs, ld, S0x, DSx, S0z, DSz, cx, cy, cz, jz, Sxi, DSzi);
      else
        deposit<T, ND, ND - 1, true>(Jx, cs, ld, S0x, DSx, S0z, DSz, cx, cy, cz, jz, Sxi, DSzi);
    } else {
      deposit<T, ND, ND, false>(Jx, cs, ld, S0x, DSx, S0z, DSz, cx, cy, cz, jz, Sxi, DSzi);
    }
    if constexpr (CP) {
      if (ion_sep) ion_jz<T, ORDER, SMEM>(Jb, cs, ld, ox, oz, is, cz);
    }
  }
  return true;
}

// current cell of a particle (grid-relative); false for a non-finite position
template <class T>
__device__ __forceinline__ bool particle_cell(const Particles<T>& p, int pi, const PushConst& pc, int& fx, int& fz) {
  if constexpr (CellPos<T>::value) {
    uint32_t c = p.cell[pi];
    float oz = p.oz[pi], ox, tz;
    if (p.w[pi] < T(0)) lattice_site_pow2(p.id[pi], pc.kb, pc.lpx, pc.lpz, pc.gx_lo, pc.z0_cells, c, ox, oz);
    fx = cell_x(c);
    frame_z(c, oz, pc.fr0_sz, pc.fr0_fz, fz, tz);
    return true;
  } else {
    const double X = p.x[pi] / pc.dx, Z = (p.z[pi] - pc.z0) / pc.dz;
    if (!(X == X) || !(Z == Z) || fabs(X) > 1e9 || fabs(Z) > 1e9) return false;
    fx = (int)floor(X); fz = (int)floor(Z);
    return true;
  }
}

// global-memory path with an index guard: a particle whose stencil would leave
// the arrays (only possible for corrupted or non-finite state) is removed and
// flagged instead of being pushed.
template <class T, int ORDER, bool MC>
__device__ __noinline__ void push_global_guarded(const T* gE, const T* gB, T* gJ, const GridP& g, const Particles<T>& p,
                                                 int pi, const PushConst& pc, Ctrl* ctrl, BoxI& acc) {
  if (p.w[pi] == T(0)) return;
  int fx, fz;
  const bool fin = particle_cell<T>(p, pi, pc, fx, fz);
  const bool ok = fin && fx >= St<ORDER>::LO + 1 && fx < g.nx - St<ORDER>::HI - 1 && fz >= St<ORDER>::LO + 1 &&
                  fz < g.nz - St<ORDER>::HI - 1;
  if (!ok) {
    p.w[pi] = T(0);
    atomicOr(&ctrl->status, fin ? ST_OUTSIDE : ST_NAN);
    return;
  }
  const Box none{0, -1, 0, -1};
  push_one<T, ORDER, false, MC>(gE, gB, gJ, g.cs, g.ld, 0, 0, p, pi, pc, none, acc);
}

// One chunk of the window kernel: stage the six gather fields of the chunk's box (+ halo) in shared memory,
// push its particles (gather, Boris, move, Esirkepov into a shared current window), add the window to J once,
// and store the box of the particles' new cells. Called by every thread of the block; s_bb is shared.
template <class T, int ORDER, bool MC>
__device__ __forceinline__ void push_chunk(const GridP& g, const T* gE, const T* gB, T* gJ, const Particles<T>& p,
                                           Chunk* chunks, Ctrl* ctrl, int cap_nodes, int tile_z,
                                           const PushDefer& pd, const PushConst& pc, int c, T* sm, int* s_bb) {
  typedef typename Vec2<T>::type V2;
  V2* smA = reinterpret_cast<V2*>(sm);                  // (Ex, Bz)
  V2* smB = reinterpret_cast<V2*>(sm + 2 * cap_nodes);  // (Ez, Bx)
  {
    const Chunk ch = chunks[c];
    const Box box{ch.ix0, ch.ix1, ch.iz0, ch.iz1};
    if (ch.ix0 > ch.ix1 || ch.p1 <= ch.p0) {   // empty chunk
      __syncthreads();
      return;
    }
    const int wx0 = ch.ix0 - St<ORDER>::LO, wx1 = ch.ix1 + St<ORDER>::HI;
    const int wz0 = ch.iz0 - St<ORDER>::LO, wz1 = ch.iz1 + St<ORDER>::HI;
    const int wxn = wx1 - wx0 + 1, wzn = wz1 - wz0 + 1;
    // A warp of a dense tile holds one particle in each of 32 consecutive cells: 32 / tile_z x-columns of
    // tile_z z-cells each. With the window's row stride congruent to tile_z modulo 32 banks, the columns'
    // 32-bit loads and atomics fall in disjoint banks; padded when the window still fits, else unpadded.
    int lds = wzn;
    if (tile_z < 32) {
      const int pad = wzn + ((tile_z - wzn) % 32 + 32) % 32;
      if (wxn * pad <= cap_nodes) lds = pad;
    }
    const int nn = wxn * lds;
    const bool use_smem = nn <= cap_nodes && wx0 >= 0 && wz0 >= 0 && wx1 <= g.nx && wz1 <= g.nz;
    typename std::conditional<CellPos<T>::value, BoxP, BoxI>::type acc;
    uint32_t* rec = reinterpret_cast<uint32_t*>(sm + 9 * cap_nodes) + threadIdx.x;   // mixed path
    if (use_smem) {
      if constexpr (CellPos<T>::value) {
        // the thread's first particle is copied while the window is staged
        if (ch.p0 + (int)threadIdx.x < ch.p1) stage_particle(p, ch.p0 + threadIdx.x, rec);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int li = e / lds, lk = e - li * lds;
        const long gp = (long)(wx0 + li) * g.ld + (wz0 + lk);
        const bool in = lk < wzn;
        T ex = T(0), ey = T(0), ez = T(0), bx = T(0), by = T(0), bz = T(0);
        if (in) {
          ex = gE[gp]; ey = gE[g.cs + gp]; ez = gE[2 * g.cs + gp];
          bx = gB[gp]; by = gB[g.cs + gp]; bz = gB[2 * g.cs + gp];
        }
        V2 va, vb;
        va.x = ex; va.y = bz;
        vb.x = ez; vb.y = bx;
        smA[e] = va;
        smB[e] = vb;
        sm[4 * cap_nodes + e] = ey;
        sm[5 * cap_nodes + e] = by;
#pragma unroll
        for (int q = 0; q < 3; q++) sm[(6 + q) * cap_nodes + e] = T(0);
      }
      __syncthreads();
      for (int pi = ch.p0 + threadIdx.x; pi < ch.p1; pi += blockDim.x) {
        const int pn = pi + blockDim.x;
        bool in_box;
        if constexpr (CellPos<T>::value) {
          // this particle's record has landed: read it, then copy the next particle into it; the xor chain
          // reads every word, so the copy is issued only once the reads have returned
          asm volatile("cp.async.wait_group 0;" ::: "memory");
          PRec r;
#pragma unroll
          for (int k = 0; k < RW_N; k++) r.v[k] = rec[k * PB_THREADS];
          uint32_t dep;
          asm volatile(
              "xor.b32 %0, %1, %2;\n\txor.b32 %0, %0, %3;\n\txor.b32 %0, %0, %4;\n\txor.b32 %0, %0, %5;\n\t"
              "xor.b32 %0, %0, %6;\n\txor.b32 %0, %0, %7;\n\txor.b32 %0, %0, %8;"
              : "=r"(dep)
              : "r"(r.v[0]), "r"(r.v[1]), "r"(r.v[2]), "r"(r.v[3]), "r"(r.v[4]), "r"(r.v[5]), "r"(r.v[6]),
                "r"(r.v[7])
              : "memory");
          (void)dep;
          if (pn < ch.p1) stage_particle(p, pn, rec);
          asm volatile("cp.async.commit_group;" ::: "memory");
          // a particle outside the chunk's box (should not happen; with electron-ion pairs, the ion's cell
          // counts too) takes the global path
          in_box = push_one<T, ORDER, true, MC, decltype(acc), true>(sm, nullptr, sm + 6 * cap_nodes, cap_nodes, lds,
                                                                     wx0, wz0, p, pi, pc, box, acc, &r);
        } else {
          // prefetch the next particle of this thread into L1
          if (pn < ch.p1) {
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.ux + pn));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.uy + pn));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.uz + pn));
            asm volatile("prefetch.global.L1 [%0];" ::"l"(p.w + pn));
          }
          in_box = push_one<T, ORDER, true, MC>(sm, nullptr, sm + 6 * cap_nodes, cap_nodes, lds, wx0, wz0, p, pi, pc,
                                                box, acc);
        }
        if (!in_box) {
          const int q = atomicAdd(&ctrl->n_defer, 1);
          if (q < pd.defer_cap) pd.defer[q] = make_int2(pi, c);
          else atomicOr(&ctrl->status, ST_OVERFLOW);
        }
      }
      if constexpr (CellPos<T>::value) asm volatile("cp.async.wait_all;" ::: "memory");
      __syncthreads();
      for (int e = threadIdx.x; e < nn; e += blockDim.x) {
        const int li = e / lds, lk = e - li * lds;
        if (lk >= wzn) continue;
        const long gp = (long)(wx0 + li) * g.ld + (wz0 + lk);
#pragma unroll
        for (int q = 0; q < 3; q++) {
          T val = sm[(6 + q) * cap_nodes + e];
          if (val != T(0)) atomicAdd(gJ + q * g.cs + gp, val);
        }
      }
    } else if (threadIdx.x == 0) {
      // the whole chunk goes to the global-memory pass; its box is rebuilt there
      atomicAdd(&ctrl->overflow_chunks, 1);
      const int q = atomicAdd(&ctrl->n_ovf, 1);
      if (q < pd.ovf_cap) pd.ovf[q] = c;
      else atomicOr(&ctrl->status, ST_OVERFLOW);
    }
    // bounding box of the chunk's live particles for the next step
    const BoxI bb = acc.unpack();
    int bx0 = bb.x0, bx1 = bb.x1, bz0 = bb.z0, bz1 = bb.z1;
    bx0 = __reduce_min_sync(0xffffffffu, bx0); bx1 = __reduce_max_sync(0xffffffffu, bx1);
    bz0 = __reduce_min_sync(0xffffffffu, bz0); bz1 = __reduce_max_sync(0xffffffffu, bz1);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&s_bb[0], bx0); atomicMax(&s_bb[1], bx1);
      atomicMin(&s_bb[2], bz0); atomicMax(&s_bb[3], bz1);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      Chunk o = ch;
      o.ix0 = s_bb[0]; o.ix1 = s_bb[1]; o.iz0 = s_bb[2]; o.iz1 = s_bb[3];
      chunks[c] = o;
    }
    __syncthreads();
  }
}

template <class T, int ORDER, bool MC>
__global__ void __launch_bounds__(PB_THREADS, 5) k_push(GridP g, const T* gE, const T* gB, T* gJ, Particles<T> p,
                                                     Chunk* chunks, Ctrl* ctrl, int cap_nodes, int tile_z,
                                                     PushDefer pd, PushConst pc) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ int s_chunk;
  __shared__ int s_bb[4];
  const int nchunks = ctrl->nchunks;
  while (true) {
    if (threadIdx.x == 0) {
      s_chunk = atomicAdd(&ctrl->next_chunk, 1);
      s_bb[0] = INT_MAX; s_bb[1] = INT_MIN; s_bb[2] = INT_MAX; s_bb[3] = INT_MIN;
    }
    __syncthreads();
    const int c = s_chunk;
    if (c >= nchunks) break;
    push_chunk<T, ORDER, MC>(g, gE, gB, gJ, p, chunks, ctrl, cap_nodes, tile_z, pd, pc, c, sm, s_bb);
  }
}

// The global-memory pass after k_push: whole chunks whose window did not fit in shared memory (one block
// each), then single particles that were outside their chunk's box (one thread each). Both add their
// current with global atomics and widen their chunk's box atomically (k_push has written the box of the
// particles it pushed; an overflow chunk's box starts empty).
template <class T, int ORDER, bool MC>
__global__ void __launch_bounds__(PB_THREADS) k_push_deferred(GridP g, const T* gE, const T* gB, T* gJ,
                                                               Particles<T> p, Chunk* chunks, Ctrl* ctrl,
                                                               PushDefer pd, PushConst pc) {
  const int novf = min(ctrl->n_ovf, pd.ovf_cap), ndef = min(ctrl->n_defer, pd.defer_cap);
  for (int j = blockIdx.x; j < novf; j += gridDim.x) {
    const int c = pd.ovf[j];
    const Chunk ch = chunks[c];
    BoxI acc;
    for (int pi = ch.p0 + threadIdx.x; pi < ch.p1; pi += blockDim.x)
      push_global_guarded<T, ORDER, MC>(gE, gB, gJ, g, p, pi, pc, ctrl, acc);
    int bx0 = acc.x0, bx1 = acc.x1, bz0 = acc.z0, bz1 = acc.z1;
    bx0 = __reduce_min_sync(0xffffffffu, bx0); bx1 = __reduce_max_sync(0xffffffffu, bx1);
    bz0 = __reduce_min_sync(0xffffffffu, bz0); bz1 = __reduce_max_sync(0xffffffffu, bz1);
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&chunks[c].ix0, bx0); atomicMax(&chunks[c].ix1, bx1);
      atomicMin(&chunks[c].iz0, bz0); atomicMax(&chunks[c].iz1, bz1);
    }
  }
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ndef; j += gridDim.x * blockDim.x) {
    const int2 e = pd.defer[j];
    BoxI acc;
    push_global_guarded<T, ORDER, MC>(gE, gB, gJ, g, p, e.x, pc, ctrl, acc);
    const int bx0 = acc.x0, bx1 = acc.x1, bz0 = acc.z0, bz1 = acc.z1;
    if (bx0 <= bx1) {
      atomicMin(&chunks[e.y].ix0, bx0); atomicMax(&chunks[e.y].ix1, bx1);
      atomicMin(&chunks[e.y].iz0, bz0); atomicMax(&chunks[e.y].iz1, bz1);
    }
  }
}

// block-wide exclusive scan of one int per thread (blockDim.x a multiple of 32, at most 1024)
__device__ int block_excl_scan(int v, int* total) {
  __shared__ int ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int s = lane < (blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  int pre = (wid > 0 ? ws[wid - 1] : 0) + x - v;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return pre;
}

// ---------------------------------------------------------------------------
// sort: tiles of tx (x) by tz (z) cells, cells numbered tile-major with z
// fastest inside a tile. Inside a tile the particles are ordered by rank in
// their cell (ranks >= R-1 share the last group), then by cell, so that a warp
// of a densely filled tile holds one particle from each of 32 consecutive
// cells: its shared-memory gathers and current atomics fall in distinct banks.
__device__ __forceinline__ int sort_cell(const SortBufs& sb, int cx, int cz) {
  const int tile = (cx / sb.tx) * sb.ntz + cz / sb.tz;
  return tile * (sb.tx * sb.tz) + (cx - (cx / sb.tx) * sb.tx) * sb.tz + (cz - (cz / sb.tz) * sb.tz);
}

template <class T>
__global__ void k_sort_key(GridP g, Particles<T> p, SortBufs sb, const Ctrl* ctrl) {
  const int n = ctrl->count;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (p.w[i] == T(0)) { sb.key[i] = -1; return; }
  int cx, cz;
  if constexpr (CellPos<T>::value) {
    uint32_t c = p.cell[i];
    float oz = p.oz[i], ox, tz;
    if (p.w[i] < T(0)) {   // ghost: its lab-fixed ion
      const uint32_t id = p.id[i];
      lattice_site((int)(id >> g.il_kb), (int)(id & ((1u << g.il_kb) - 1u)), g.il_ppcx, g.il_ppcz, g.gx_lo,
                   g.z0_cells, c, ox, oz);
    }
    cx = cell_x(c);
    frame_z(c, oz, g.fr_sz, g.fr_fz, cz, tz);
  } else {
    cx = (int)floor(p.x[i] / g.dx);
    cz = (int)floor((p.z[i] - g.z0) / g.dz);
  }
  cx = min(max(cx, 0), g.nx - 1);
  cz = min(max(cz, 0), g.nz - 1);
  const int c = sort_cell(sb, cx, cz);
  sb.key[i] = c;
  sb.slot[i] = atomicAdd(&sb.cell_cnt[c], 1);
}

// particles per tile (one block per tile, one thread per cell; tiles of up to 1024 cells)
__global__ void __launch_bounds__(1024) k_tile_count(SortBufs sb) {
  const int tc = sb.tx * sb.tz;
  const int cl = threadIdx.x;
  int v = cl < tc ? sb.cell_cnt[(long)blockIdx.x * tc + cl] : 0;
  int total;
  block_excl_scan(v, &total);
  if (threadIdx.x == 0) sb.tile_cnt[blockIdx.x] = total;
}

// destination of every (cell, rank) entry of a tile (one block per tile, one thread per cell)
__global__ void __launch_bounds__(1024) k_tile_order(SortBufs sb) {
  const int tc = sb.tx * sb.tz;
  const int cl = threadIdx.x;
  const long c = (long)blockIdx.x * tc + cl;
  const int cnt = cl < tc ? sb.cell_cnt[c] : 0;
  const int base = sb.tile_start[blockIdx.x];
  int tot;
  const int cstart = base + block_excl_scan(cnt, &tot);
  if (cl < tc) sb.cell_start[c] = cstart;
  int off = base;
  int r = 0;
  for (; r < sb.R - 1; r++) {
    const int f = cnt > r;
    if (!__syncthreads_or(f)) break;
    int tr;
    const int pos = block_excl_scan(f, &tr);
    if (f) sb.dest[cstart + r] = off + pos;
    off += tr;
  }
  // ranks >= R-1: the rest of each cell, cell after cell
  const int m = r == sb.R - 1 ? max(cnt - r, 0) : 0;
  if (__syncthreads_or(m > 0)) {
    int tm;
    const int pos = block_excl_scan(m, &tm);
    for (int j = 0; j < m; j++) sb.dest[cstart + r + j] = off + pos + j;
  }
}

template <class T>
__global__ void k_sort_scatter(Particles<T> s, Particles<T> d, SortBufs sb, const Ctrl* ctrl) {
  const int n = ctrl->count;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int key = sb.key[i];
  if (key < 0) return;
  const int o = sb.dest[sb.cell_start[key] + sb.slot[i]];
  if constexpr (CellPos<T>::value) {
    d.cell[o] = s.cell[i]; d.ox[o] = s.ox[i]; d.oz[o] = s.oz[i];
  } else {
    d.x[o] = s.x[i]; d.z[o] = s.z[i];
  }
  d.ux[o] = s.ux[i]; d.uy[o] = s.uy[i]; d.uz[o] = s.uz[i];
  d.w[o] = s.w[i]; d.id[o] = s.id[i];
}

__global__ void k_build_chunks(SortBufs sb, Chunk* chunks, Ctrl* ctrl, int chunk_max, int chunk_cap, int nx, int nz) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ntiles = sb.ntx * sb.ntz;
  if (t >= ntiles) return;
  const int p0 = sb.tile_start[t], p1 = sb.tile_start[t + 1];
  const int n = p1 - p0;
  if (n <= 0) return;
  const int nch = (n + chunk_max - 1) / chunk_max;
  const int base = atomicAdd(&ctrl->nchunks, nch);
  const int tx = t / sb.ntz, tz = t - tx * sb.ntz;
  for (int j = 0; j < nch; j++) {
    if (base + j >= chunk_cap) { atomicOr(&ctrl->status, ST_OVERFLOW); return; }
    Chunk c;
    c.p0 = p0 + j * chunk_max;
    c.p1 = min(p1, p0 + (j + 1) * chunk_max);
    c.ix0 = tx * sb.tx; c.ix1 = min(nx - 1, (tx + 1) * sb.tx - 1);
    c.iz0 = tz * sb.tz; c.iz1 = min(nz - 1, (tz + 1) * sb.tz - 1);
    chunks[base + j] = c;
  }
}

__global__ void k_sort_finish_pre(Ctrl* ctrl) { ctrl->nchunks = 0; }
__global__ void k_sort_finish(Ctrl* ctrl, const int* bin_start, int nbins) { ctrl->count = bin_start[nbins]; }

// exclusive scan of n ints (n <= 1024*1024): block sums, scan of sums, local scans
__global__ void k_scan_sums(const int* in, int n, int* sums) {
  __shared__ int ws[32];
  const int i = blockIdx.x * 1024 + threadIdx.x;
  int v = i < n ? in[i] : 0;
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int s = ws[threadIdx.x];
    s = __reduce_add_sync(0xffffffffu, s);
    if (threadIdx.x == 0) sums[blockIdx.x] = s;
  }
}

__global__ void k_scan_top(int* sums, int nb) {
  // single block of 1024 threads; nb <= 1024
  int v = threadIdx.x < nb ? sums[threadIdx.x] : 0;
  int pre = block_excl_scan(v, nullptr);
  if (threadIdx.x < nb) sums[threadIdx.x] = pre;
}

__global__ void k_scan_local(const int* in, int n, const int* sums, int* out) {
  const int i = blockIdx.x * 1024 + threadIdx.x;
  int v = i < n ? in[i] : 0;
  int total;
  int pre = block_excl_scan(v, &total);
  const int off = sums[blockIdx.x];
  if (i < n) out[i] = off + pre;
  if (i == n - 1) out[n] = off + pre + v;
}

// ---------------------------------------------------------------------------
// plasma rows entering through the plane z_hi (or the initial load)
__device__ double lab_density(const InjectP& ip, double zl) {
  if (zl < ip.z_start_lab) return 0.0;
  double r = zl - ip.z_start_lab;
  if (ip.ramp_lab > 0.0 && r < ip.ramp_lab) return ip.n0 * r / ip.ramp_lab;
  double pe = ip.ramp_lab + ip.length_lab;
  if (ip.length_lab > 0.0 && r >= pe) return 0.0;
  return ip.n0;
}

template <class T>
__device__ __forceinline__ void inject_block(const GridP& g, const Particles<T>& p, Chunk* chunks, Ctrl* ctrl,
                                             const InjectP& ip, int cap, int chunk_cap, int xb, int rb, int nxb) {
  const long long nrows = ip.m_end - ip.m_beg;
  const long long r0 = (long long)rb * ip.rblock;
  const int nr = (int)min((long long)ip.rblock, nrows - r0);
  const int ncx_dom = g.gx_hi - g.gx_lo;
  const int cx0 = xb * ip.xblock;
  const int ncx = min(ip.xblock, ncx_dom - cx0);
  const int per_row = ncx * ip.ppc_x;
  const int cnt = nr * per_row;
  const int base = ctrl->count;
  const long long start = (long long)base + r0 * ip.nxl + (long long)nr * cx0 * ip.ppc_x;
  const double gdz = g.dz;
  for (int j = threadIdx.x; j < cnt; j += blockDim.x) {
    const int r = j / per_row, al = j - r * per_row;
    const long long m = ip.m_beg + r0 + r;
    const long long a = (long long)cx0 * ip.ppc_x + al;
    const long long o = start + j;
    if (o >= cap) { atomicOr(&ctrl->status, ST_OVERFLOW); continue; }
    const double zlat = (m + 0.5) * ip.h;
    const double n = ip.gamma * lab_density(ip, ip.gamma * zlat);
    const double zp = zlat - ip.beta * kC * ip.t;
    if constexpr (CellPos<T>::value) {
      // drifting frame: the row's lattice position (grid z + beta c t / dz)
      uint32_t c;
      float sox, soz;
      lattice_site((int)m, (int)a, ip.ppc_x, ip.ppc_z, g.gx_lo, g.z0_cells, c, sox, soz);
      p.cell[o] = c;
      p.ox[o] = sox;
      p.oz[o] = soz;
    } else {
      p.x[o] = (g.gx_lo + (a + 0.5) / ip.ppc_x) * g.dx;
      p.z[o] = zp;
    }
    p.ux[o] = T(0); p.uy[o] = T(0);
    // mixed path: the deviation from the drift momentum, which it starts at
    p.uz[o] = CellPos<T>::value ? T(0) : T(-ip.gamma * ip.beta * kC);
    p.w[o] = T(n * g.dx * gdz / (double)(ip.ppc_x * ip.ppc_z));
    if constexpr (CellPos<T>::value) p.id[o] = ((uint32_t)m << g.il_kb) | (uint32_t)a;
    else p.id[o] = (uint32_t)((unsigned long long)m * (unsigned long long)ip.nxl + (unsigned long long)a);
  }
  if (threadIdx.x == 0 && cnt > 0) {
    const int ci = ctrl->nchunks + rb * nxb + xb;
    if (ci >= chunk_cap || start + cnt > cap) { atomicOr(&ctrl->status, ST_OVERFLOW); return; }
    Chunk c;
    c.p0 = (int)start; c.p1 = (int)(start + cnt);
    c.ix0 = g.gx_lo + cx0; c.ix1 = g.gx_lo + cx0 + ncx - 1;
    const double za = ((ip.m_beg + r0 + 0.5) * ip.h - ip.beta * kC * ip.t - g.z0) / gdz;
    const double zb = ((ip.m_beg + r0 + nr - 1 + 0.5) * ip.h - ip.beta * kC * ip.t - g.z0) / gdz;
    c.iz0 = (int)floor(za); c.iz1 = (int)floor(zb);
    chunks[ci] = c;
  }
}

template <class T>
__global__ void k_inject(GridP g, Particles<T> p, Chunk* chunks, Ctrl* ctrl, InjectP ip, int cap, int chunk_cap) {
  inject_block<T>(g, p, chunks, ctrl, ip, cap, chunk_cap, blockIdx.x, blockIdx.y, gridDim.x);
}

__global__ void k_add_counts(Ctrl* ctrl, int dcount, int dchunks) {
  ctrl->count += dcount;
  ctrl->nchunks += dchunks;
}

// ---------------------------------------------------------------------------
// batched particle kernels of an ensemble step
constexpr int MAX_BATCH_RUNS = 512;

template <class T>
__global__ void k_push_batch_reset(const StepArgs<T>* a, int nruns, int* counter) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r == 0) *counter = 0;
  if (r < nruns && a[r].push_on) { a[r].ctrl->n_defer = 0; a[r].ctrl->n_ovf = 0; }
}

// the window kernel over all runs' chunks: blocks take (run, chunk) pairs from one queue; the run's push
// constants, geometry and particle arrays are copied to shared memory when a block changes run
template <class T, int ORDER>
__global__ void __launch_bounds__(PB_THREADS, 5) k_push_batch(const StepArgs<T>* a, int nruns, int* counter,
                                                           int cap_nodes, int tile_z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* sm = reinterpret_cast<T*>(smraw);
  __shared__ int s_pref[MAX_BATCH_RUNS + 1];
  __shared__ int s_w, s_r, s_bb[4];
  __shared__ PushConst s_pc;
  __shared__ GridP s_g;
  __shared__ Particles<T> s_p;
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < nruns; r++) {
      s_pref[r] = acc;
      if (a[r].push_on) acc += a[r].ctrl->nchunks;
    }
    s_pref[nruns] = acc;
  }
  __syncthreads();
  const int total = s_pref[nruns];
  int cur = -1;
  while (true) {
    if (threadIdx.x == 0) {
      const int w = atomicAdd(counter, 1);
      s_w = w;
      if (w < total) {
        int lo = 0, hi = nruns - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_pref[mid] <= w) lo = mid;
          else hi = mid - 1;
        }
        s_r = lo;
      }
      s_bb[0] = INT_MAX; s_bb[1] = INT_MIN; s_bb[2] = INT_MAX; s_bb[3] = INT_MIN;
    }
    __syncthreads();
    const int w = s_w;
    if (w >= total) break;
    const int r = s_r;
    if (r != cur) {
      if (threadIdx.x == 0) { s_pc = a[r].pc; s_g = a[r].g; s_p = a[r].p; }
      __syncthreads();
      cur = r;
    }
    const StepArgs<T>& A = a[r];
    push_chunk<T, ORDER, false>(s_g, A.f.fE[0], A.f.fB[0], A.f.J[0], s_p, A.chunks, A.ctrl, cap_nodes, tile_z, A.pd,
                                s_pc, w - s_pref[r], sm, s_bb);
  }
}

// the global-memory pass of every run (usually nothing to do)
template <class T, int ORDER>
__global__ void __launch_bounds__(PB_THREADS) k_push_deferred_batch(const StepArgs<T>* a, int nruns) {
  for (int r = 0; r < nruns; r++) {
    const StepArgs<T>& A = a[r];
    if (!A.push_on) continue;
    const int novf = min(A.ctrl->n_ovf, A.pd.ovf_cap), ndef = min(A.ctrl->n_defer, A.pd.defer_cap);
    for (int j = blockIdx.x; j < novf; j += gridDim.x) {
      const int c = A.pd.ovf[j];
      const Chunk ch = A.chunks[c];
      BoxI acc;
      for (int pi = ch.p0 + threadIdx.x; pi < ch.p1; pi += blockDim.x)
        push_global_guarded<T, ORDER, false>(A.f.fE[0], A.f.fB[0], A.f.J[0], A.g, A.p, pi, A.pc, A.ctrl, acc);
      int bx0 = acc.x0, bx1 = acc.x1, bz0 = acc.z0, bz1 = acc.z1;
      bx0 = __reduce_min_sync(0xffffffffu, bx0); bx1 = __reduce_max_sync(0xffffffffu, bx1);
      bz0 = __reduce_min_sync(0xffffffffu, bz0); bz1 = __reduce_max_sync(0xffffffffu, bz1);
      if ((threadIdx.x & 31) == 0) {
        atomicMin(&A.chunks[c].ix0, bx0); atomicMax(&A.chunks[c].ix1, bx1);
        atomicMin(&A.chunks[c].iz0, bz0); atomicMax(&A.chunks[c].iz1, bz1);
      }
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < ndef; j += gridDim.x * blockDim.x) {
      const int2 e = A.pd.defer[j];
      BoxI acc;
      push_global_guarded<T, ORDER, false>(A.f.fE[0], A.f.fB[0], A.f.J[0], A.g, A.p, e.x, A.pc, A.ctrl, acc);
      const int bx0 = acc.x0, bx1 = acc.x1, bz0 = acc.z0, bz1 = acc.z1;
      if (bx0 <= bx1) {
        atomicMin(&A.chunks[e.y].ix0, bx0); atomicMax(&A.chunks[e.y].ix1, bx1);
        atomicMin(&A.chunks[e.y].iz0, bz0); atomicMax(&A.chunks[e.y].iz1, bz1);
      }
    }
  }
}

// plasma rows entering every run this step: blocks (x-block, row-block) of each run, those past the
// run's rows idle
template <class T>
__global__ void k_inject_batch(const StepArgs<T>* a, const int* off, int nruns) {
  __shared__ int s_r;
  if (threadIdx.x == 0) s_r = batch_run(off, nruns, blockIdx.x);
  __syncthreads();
  const StepArgs<T>& A = a[s_r];
  if (!A.inj_on) return;
  const int lb = blockIdx.x - off[s_r];
  const int xb = lb % A.inj_xblocks, rb = lb / A.inj_xblocks;
  if ((long long)rb * A.ip.rblock >= A.ip.m_end - A.ip.m_beg) return;
  inject_block<T>(A.g, A.p, A.chunks, A.ctrl, A.ip, A.cap, A.chunk_cap, xb, rb, A.inj_xblocks);
}

template <class T>
__global__ void k_add_counts_batch(const StepArgs<T>* a, int nruns) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nruns && a[r].inj_on) {
    a[r].ctrl->count += a[r].add_count;
    a[r].ctrl->nchunks += a[r].add_chunks;
  }
}

}  // namespace

template <class T>
void launch_push_batch(const StepArgs<T>* a, const BatchGrid& bg, int order, int grid_blocks, int smem_nodes,
                       int tile_z, cudaStream_t s) {
  const size_t sm = (size_t)9 * smem_nodes * sizeof(T) + push_stage_bytes<T>();
  k_push_batch_reset<T><<<(bg.nruns + 255) / 256, 256, 0, s>>>(a, bg.nruns, bg.push_counter);
  const int gb = grid_blocks < 304 ? grid_blocks : 304;
  if (order == 3) {
    cudaFuncSetAttribute(k_push_batch<T, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push_batch<T, 3><<<grid_blocks, PB_THREADS, sm, s>>>(a, bg.nruns, bg.push_counter, smem_nodes, tile_z);
    k_push_deferred_batch<T, 3><<<gb, PB_THREADS, 0, s>>>(a, bg.nruns);
  } else {
    cudaFuncSetAttribute(k_push_batch<T, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push_batch<T, 1><<<grid_blocks, PB_THREADS, sm, s>>>(a, bg.nruns, bg.push_counter, smem_nodes, tile_z);
    k_push_deferred_batch<T, 1><<<gb, PB_THREADS, 0, s>>>(a, bg.nruns);
  }
}

template <class T>
void launch_inject_batch(const StepArgs<T>* a, const BatchGrid& bg, cudaStream_t s) {
  k_inject_batch<T><<<bg.inj_blocks, 256, 0, s>>>(a, bg.inj_off, bg.nruns);
  k_add_counts_batch<T><<<(bg.nruns + 127) / 128, 128, 0, s>>>(a, bg.nruns);
}

PushConst push_const(const GridP& g, double q, double m, double gamma_b, int fr1_sz, float fr1_fz, int pairs,
                     int mlo) {
  PushConst pc;
  pc.dx = g.dx; pc.dz = g.dz; pc.dt = g.dt; pc.z0 = g.z0;
  pc.xlo = g.gx_lo * g.dx; pc.xhi = g.gx_hi * g.dx;
  pc.zlo = g.z0 + g.gz_lo * g.dz; pc.zhi = g.z0 + g.gz_hi * g.dz + g.dz;
  pc.cx_lo = g.gx_lo; pc.cx_hi = g.gx_hi; pc.cz_lo = g.gz_lo; pc.cz_hi = g.gz_hi + 1;
  pc.dtdx = (float)(g.dt / g.dx); pc.dtdz = (float)(g.dt / g.dz);
  pc.qm_half = q * g.dt / (2.0 * m);
  pc.kx = -q / (g.dz * g.dt); pc.kz = -q / (g.dx * g.dt); pc.ky = q / (g.dx * g.dz);
  pc.qm_half_f = (float)pc.qm_half; pc.kx_f = (float)pc.kx; pc.kz_f = (float)pc.kz; pc.ky_f = (float)pc.ky;
  pc.u0z_f = g.fr_u0;
  pc.g0_f = (float)gamma_b;
  pc.g0sq_f = (float)(1.0 + (double)g.fr_u0 * (double)g.fr_u0 / (kC * kC));
  pc.fr0_sz = g.fr_sz; pc.fr0_fz = g.fr_fz;
  pc.fr1_sz = fr1_sz; pc.fr1_fz = fr1_fz;
  pc.pairs = pairs; pc.mlo = mlo;
  pc.kb = g.il_kb; pc.gx_lo = g.gx_lo; pc.z0_cells = g.z0_cells;
  pc.lpx = 0; pc.lpz = 0;
  while ((1 << pc.lpx) < g.il_ppcx) pc.lpx++;
  while ((1 << pc.lpz) < g.il_ppcz) pc.lpz++;
  return pc;
}

template <class T>
void launch_push(const GridP& g, const FieldPtrs<T>& f, Particles<T> p, Chunk* chunks, Ctrl* ctrl, int order,
                 int grid_blocks, int smem_nodes, int tile_z, double q, double m, double gamma_b, double beta_b,
                 int fr1_sz, float fr1_fz, int pairs, int mlo, int nodal, const PushDefer& pd, cudaStream_t s) {
  (void)beta_b;
  const PushConst pc = push_const(g, q, m, gamma_b, fr1_sz, fr1_fz, pairs, mlo);
  const size_t sm = (size_t)9 * smem_nodes * sizeof(T) + push_stage_bytes<T>();
  cudaMemsetAsync(&ctrl->next_chunk, 0, sizeof(int), s);
  cudaMemsetAsync(&ctrl->n_defer, 0, 2 * sizeof(int), s);
  // 'momentum conserving' gather: the node-interpolated copies; else the Yee-located gather copies
  const T* gE = nodal ? f.nE[0] : f.fE[0];
  const T* gB = nodal ? f.nB[0] : f.fB[0];
  if (order == 3 && !nodal) {
    cudaFuncSetAttribute(k_push<T, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push<T, 3, false><<<grid_blocks, PB_THREADS, sm, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, smem_nodes, tile_z, pd, pc);
  } else if (order == 3) {
    cudaFuncSetAttribute(k_push<T, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push<T, 3, true><<<grid_blocks, PB_THREADS, sm, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, smem_nodes, tile_z, pd, pc);
  } else if (!nodal) {
    cudaFuncSetAttribute(k_push<T, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push<T, 1, false><<<grid_blocks, PB_THREADS, sm, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, smem_nodes, tile_z, pd, pc);
  } else {
    cudaFuncSetAttribute(k_push<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_push<T, 1, true><<<grid_blocks, PB_THREADS, sm, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, smem_nodes, tile_z, pd, pc);
  }
  // the global-memory pass over what the window kernel left (usually nothing: the blocks exit at once)
  const int gb = grid_blocks < 304 ? grid_blocks : 304;
  if (order == 3 && !nodal) k_push_deferred<T, 3, false><<<gb, PB_THREADS, 0, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, pd, pc);
  else if (order == 3) k_push_deferred<T, 3, true><<<gb, PB_THREADS, 0, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, pd, pc);
  else if (!nodal) k_push_deferred<T, 1, false><<<gb, PB_THREADS, 0, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, pd, pc);
  else k_push_deferred<T, 1, true><<<gb, PB_THREADS, 0, s>>>(g, gE, gB, f.J[0], p, chunks, ctrl, pd, pc);
}

int push_occupancy(int order, bool dbl, int smem_nodes) {
  int nb = 0;
  if (dbl) {
    size_t sm = (size_t)9 * smem_nodes * sizeof(double);
    if (order == 3) {
      cudaFuncSetAttribute(k_push<double, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<double, 3, false>, PB_THREADS, sm);
    } else {
      cudaFuncSetAttribute(k_push<double, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<double, 1, false>, PB_THREADS, sm);
    }
  } else {
    size_t sm = (size_t)9 * smem_nodes * sizeof(float) + push_stage_bytes<float>();
    if (order == 3) {
      cudaFuncSetAttribute(k_push<float, 3, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<float, 3, false>, PB_THREADS, sm);
    } else {
      cudaFuncSetAttribute(k_push<float, 1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_push<float, 1, false>, PB_THREADS, sm);
    }
  }
  return nb > 0 ? nb : 1;
}

static void exclusive_scan(const int* in, int n, int* out, int* tmp, cudaStream_t s) {
  const int nb = (n + 1023) / 1024;
  k_scan_sums<<<nb, 1024, 0, s>>>(in, n, tmp);
  k_scan_top<<<1, 1024, 0, s>>>(tmp, nb);
  k_scan_local<<<nb, 1024, 0, s>>>(in, n, tmp, out);
}

template <class T>
void launch_sort(const GridP& g, Particles<T> src, Particles<T> dst, SortBufs sb, Chunk* chunks, Ctrl* ctrl, int cap,
                 int chunk_max, int chunk_cap, cudaStream_t s) {
  const int ntiles = sb.ntx * sb.ntz;
  const int tc = sb.tx * sb.tz;
  const int tb = (tc + 31) / 32 * 32;   // one thread per cell of a tile
  cudaMemsetAsync(sb.cell_cnt, 0, sizeof(int) * (size_t)ntiles * tc, s);
  const int nb = (cap + 255) / 256;
  k_sort_key<T><<<nb, 256, 0, s>>>(g, src, sb, ctrl);
  k_tile_count<<<ntiles, tb, 0, s>>>(sb);
  exclusive_scan(sb.tile_cnt, ntiles, sb.tile_start, sb.scan_tmp, s);
  k_tile_order<<<ntiles, tb, 0, s>>>(sb);
  k_sort_scatter<T><<<nb, 256, 0, s>>>(src, dst, sb, ctrl);
  k_sort_finish_pre<<<1, 1, 0, s>>>(ctrl);
  k_build_chunks<<<(ntiles + 255) / 256, 256, 0, s>>>(sb, chunks, ctrl, chunk_max, chunk_cap, g.nx, g.nz);
  k_sort_finish<<<1, 1, 0, s>>>(ctrl, sb.tile_start, ntiles);
}

template <class T>
void launch_inject(const GridP& g, Particles<T> p, Chunk* chunks, Ctrl* ctrl, const InjectP& ip, int cap,
                   int chunk_cap, cudaStream_t s) {
  const long long nrows = ip.m_end - ip.m_beg;
  if (nrows <= 0) return;
  const int ncx = g.gx_hi - g.gx_lo;
  dim3 grd((ncx + ip.xblock - 1) / ip.xblock, (unsigned)((nrows + ip.rblock - 1) / ip.rblock));
  k_inject<T><<<grd, 256, 0, s>>>(g, p, chunks, ctrl, ip, cap, chunk_cap);
  launch_add_counts(ctrl, (int)(nrows * ip.nxl), (int)(grd.x * grd.y), s);
}

void launch_add_counts(Ctrl* ctrl, int dcount, int dchunks, cudaStream_t s) {
  k_add_counts<<<1, 1, 0, s>>>(ctrl, dcount, dchunks);
}

#define INST(T)                                                                                                 \
  template void launch_push<T>(const GridP&, const FieldPtrs<T>&, Particles<T>, Chunk*, Ctrl*, int, int, int,   \
                               int, double, double, double, double, int, float, int, int, int, const PushDefer&, \
                               cudaStream_t);                                                                   \
  template void launch_sort<T>(const GridP&, Particles<T>, Particles<T>, SortBufs, Chunk*, Ctrl*, int, int, int,\
                               cudaStream_t);                                                                   \
  template void launch_inject<T>(const GridP&, Particles<T>, Chunk*, Ctrl*, const InjectP&, int, int, cudaStream_t); \
  template void launch_push_batch<T>(const StepArgs<T>*, const BatchGrid&, int, int, int, int, cudaStream_t);      \
  template void launch_inject_batch<T>(const StepArgs<T>*, const BatchGrid&, cudaStream_t);
INST(float)
INST(double)
#undef INST

}  // namespace picgb
