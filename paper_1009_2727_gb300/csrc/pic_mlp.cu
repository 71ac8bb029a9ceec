// Multilayer perceptron for the stage surrogate: widths w0 -> w1 -> ... -> wL,
// GELU between layers and a linear output. Weights are kept as FP32 master
// copies (AdamW) and BF16 compute copies; activations are stored in BF16; every
// product accumulates in FP32. One tiled GEMM kernel serves the forward pass
// (X W^T), the weight gradient (dZ^T H) and the input gradient (dZ W).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <vector>

#include "../../include/pic.h"

namespace {

constexpr int GT = 64;    // output tile (rows and columns)
constexpr int GK = 16;    // reduction slice

__device__ __forceinline__ float ld_el(const float* p, long i) { return p[i]; }
__device__ __forceinline__ float ld_el(const __nv_bfloat16* p, long i) { return __bfloat162float(p[i]); }

// C(m, n) = sum_k A(m, k) B(k, n) (+ bias[n]); A(m, k) = TA ? A[k lda + m] : A[m lda + k],
// B(k, n) = TB ? B[n ldb + k] : B[k ldb + n]. 256 threads, 64 x 64 tile, 4 x 4 outputs per thread.
// EPI 0: store C (FP32); EPI 1: store Z = C + bias (FP32) and H = GELU(Z) (BF16); EPI 2: store C + bias.
template <class TAe, class TBe, bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const TAe* A, int lda, const TBe* B, int ldb,
                                              float* C, int ldc, const float* bias, __nv_bfloat16* H) {
  __shared__ float As[GK][GT + 1];
  __shared__ float Bs[GK][GT + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GK * GT; e += 256) {
      const int kk = e / GT, mm = e - kk * GT;
      const int m = m0 + mm, n = n0 + mm, k = k0 + kk;
      float a = 0.0f, b = 0.0f;
      if (m < M && k < K) a = TA ? ld_el(A, (long)k * lda + m) : ld_el(A, (long)m * lda + k);
      if (n < N && k < K) b = TB ? ld_el(B, (long)n * ldb + k) : ld_el(B, (long)k * ldb + n);
      As[kk][mm] = a;
      Bs[kk][mm] = b;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk++) {
      float av[4], bv[4];
#pragma unroll
      for (int i = 0; i < 4; i++) { av[i] = As[kk][ty + 16 * i]; bv[i] = Bs[kk][tx + 16 * i]; }
#pragma unroll
      for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] += av[i] * bv[j];
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; i++)
#pragma unroll
    for (int j = 0; j < 4; j++) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m >= M || n >= N) continue;
      float v = acc[i][j];
      if (EPI >= 1) v += bias[n];
      C[(long)m * ldc + n] = v;
      if (EPI == 1) H[(long)m * ldc + n] = __float2bfloat16(0.5f * v * (1.0f + erff(v * 0.70710678118654752f)));
    }
}

// dZ = dH * GELU'(Z), GELU'(z) = Phi(z) + z phi(z)
__global__ void k_gelu_back(long n, const float* Z, const float* dH, float* dZ) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float z = Z[i];
  const float d = 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
  dZ[i] = dH[i] * d;
}

// db[j] = sum_i dZ[i, j] (one block per column)
__global__ void k_colsum(int n, int cols, const float* dZ, float* db) {
  __shared__ float red[256];
  const int j = blockIdx.x;
  float s = 0.0f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += dZ[(long)i * cols + j];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[j] = red[0];
}

// mean squared error over n x d outputs; dY = 2 (Y - T) / (n d); loss summed into *loss
// loss: the sum is added to loss[*eidx] when eidx is given (the epoch's slot of a training run), else to *loss
__global__ void k_mse(long nd, const float* Y, const float* T, float* dY, float* loss, const int* eidx) {
  __shared__ float red[256];
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.0f;
  if (i < nd) {
    const float e = Y[i] - T[i];
    dY[i] = 2.0f * e / (float)nd;
    l = e * e / (float)nd;
  }
  red[threadIdx.x] = l;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(eidx ? loss + *eidx : loss, red[0]);
}

__global__ void k_to_bf16(long n, const float* src, __nv_bfloat16* dst) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// AdamW (decoupled weight decay) on the FP32 master parameters, then their BF16 copies. The bias corrections
// c1 = 1 - b1^t, c2 = 1 - b2^t come as arguments, or (ctab given) from a host-computed table at step
// (*eidx) * nbat + kk: the form a captured epoch replays
__global__ void k_adamw(long n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float b1,
                        float b2, float eps, float wd, float c1, float c2, const float2* ctab, const int* eidx,
                        int nbat, int kk) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (ctab) {
    const float2 c = ctab[(long)(*eidx) * nbat + kk];
    c1 = c.x;
    c2 = c.y;
  }
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + wd * p[i]);
  p[i] = pi;
  pb[i] = __float2bfloat16(pi);
}

// rows idx[i] of X (n x dx) and T (n x dt) into contiguous batches
__global__ void k_gather_rows(int nb, const int* idx, const float* X, int dx, const float* T, int dt, float* Xb,
                              float* Tb) {
  const int r = blockIdx.x;
  if (r >= nb) return;
  const long s = idx[r];
  for (int j = threadIdx.x; j < dx; j += blockDim.x) Xb[(long)r * dx + j] = X[s * dx + j];
  for (int j = threadIdx.x; j < dt; j += blockDim.x) Tb[(long)r * dt + j] = T[s * dt + j];
}

uint64_t splitmix64(uint64_t& s) {
  uint64_t z = (s += 0x9e3779b97f4a7c15ULL);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

// ---------------------------------------------------------------------------
// Tensor-core inference (tcgen05): one CTA takes 128 rows through every layer. Each layer's weights
// come as a prepacked BF16 image (K-major, no swizzle, padded to multiples of 16) by one bulk TMA copy
// into shared memory; the activations of the 128 rows sit in shared memory in the same canonical layout;
// one thread issues the K/16 tcgen05.mma (M = 128, N = padded width, BF16 x BF16 -> FP32) into a TMEM
// accumulator; the four warps read their 32 TMEM lanes (one row per thread), add the bias, apply GELU
// and write the next layer's operand (or the FP32 outputs) in place.
constexpr int TC_M = 128;
constexpr int TC_THREADS = 512;                            // 16 warps: 4 TMEM lane groups x 4 column groups
constexpr int TC_MAXW = 256;                              // padded width limit of this kernel
constexpr int TC_A_BYTES = TC_M * TC_MAXW * 2;            // activations
constexpr int TC_B_BYTES = TC_MAXW * TC_MAXW * 2;         // one layer's weights
constexpr int TC_SMEM = TC_A_BYTES + TC_B_BYTES + 64;
constexpr int TC_MAXL = 16;

__host__ __device__ inline int pad16(int v) { return (v + 15) & ~15; }

// byte offset of element (r, k) of an operand with Kp columns: 8 x 8 core matrices of 128 contiguous
// bytes (a row of 8 elements every 16 bytes), K-groups 128 bytes apart, 8-row groups Kp * 16 bytes apart
__host__ __device__ inline uint32_t canon_off(int r, int k, int Kp) {
  return (uint32_t)((r >> 3) * (Kp * 16) + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__global__ void k_next_epoch(int* eidx) { *eidx += 1; }

__global__ void k_pack_weights(const __nv_bfloat16* W, int N, int K, int Np, int Kp, __nv_bfloat16* img) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= Np * Kp) return;
  const int r = e / Kp, k = e - r * Kp;
  img[canon_off(r, k, Kp) >> 1] = (r < N && k < K) ? W[(long)r * K + k] : __float2bfloat16(0.0f);
}

struct TcLayer {
  const __nv_bfloat16* img;
  const float* bias;
  int N, K, Np, Kp;
};
struct TcNet {
  TcLayer l[TC_MAXL];
  int L, k0;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO (K direction), SBO (8-row groups), fixed version bits 46-47,
// no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// wait for the phase of an mbarrier, giving up after about half a second (then the error flag is set)
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  const uint64_t t0 = global_ns();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > 500000000ull) {
      atomicExch(err, 1);
      return false;
    }
  }
}

// erf by Abramowitz & Stegun, Handbook of Mathematical Functions, 7.1.26 (Hastings' rational
// approximation; |error| <= 1.5e-7 for x >= 0, far below the BF16 rounding that every activation takes):
// erf(x) = 1 - t (a1 + a2 t + a3 t^2 + a4 t^3 + a5 t^4) exp(-x^2), t = 1 / (1 + p x), odd in x.
// About half the instructions of the library erf in the serving epilogue, which bounds the kernel.
__device__ __forceinline__ float erf_as(float x) {
  const float ax = fabsf(x);
  const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
  const float poly =
      t * fmaf(fmaf(fmaf(fmaf(1.061405429f, t, -1.453152027f), t, 1.421413741f), t, -0.284496736f), t,
               0.254829592f);
  return copysignf(fmaf(-poly, __expf(-ax * ax), 1.0f), x);
}

// exact (erf-form) GELU of the serving path
__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erf_as(z * 0.70710678118654752f)); }

__global__ void __launch_bounds__(TC_THREADS, 1) k_mlp_fwd_tc(TcNet net, const float* __restrict__ x, long n,
                                                             float* __restrict__ y, int* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* A = sm;
  unsigned char* Bw = sm + TC_A_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TC_A_BYTES + TC_B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // TMEM lanes 32 (warp % 4) .. +31 are this warp's rows; chunks of 16 columns go round-robin to warp / 4
  const int lgrp = warp & 3, cgrp = warp >> 2;
  const int rloc = lgrp * 32 + lane;
  const long row0 = (long)blockIdx.x * TC_M;
  const uint32_t barW = smem_u32(&bars[0]), barM = smem_u32(&bars[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barW) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(barM) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // the 128 input rows, BF16, zero padded, in the first layer's operand layout
  {
    const int Kp = net.l[0].Kp, nk8 = Kp / 8;
    for (int e = tid; e < TC_M * nk8; e += TC_THREADS) {
      const int rr = e / nk8, k8 = e - rr * nk8;
      const long r = row0 + rr;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int q = 0; q < 8; q++) {
        const int k = k8 * 8 + q;
        v[q] = __float2bfloat16((r < n && k < net.k0) ? x[r * net.k0 + k] : 0.0f);
      }
      *reinterpret_cast<uint4*>(A + canon_off(rr, k8 * 8, Kp)) = *reinterpret_cast<const uint4*>(v);
    }
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  uint32_t phW = 0, phM = 0;
  bool ok = true;
  // the weights of layer l arrive by one bulk copy, issued for the next layer as soon as the current
  // layer's products have completed (it overlaps the epilogue)
  auto load_weights = [&](int l) {
    const uint32_t bytes = (uint32_t)(net.l[l].Np * net.l[l].Kp * 2);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(barW), "r"(bytes) : "memory");
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(Bw)),
                 "l"(net.l[l].img), "r"(bytes), "r"(barW)
                 : "memory");
  };
  if (tid == 0) load_weights(0);
  for (int l = 0; l < net.L; l++) {
    const TcLayer Ly = net.l[l];
    ok = __syncthreads_and(mbar_wait(barW, phW, err) ? 1 : 0) != 0;
    phW ^= 1u;
    if (!ok) break;
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Ly.Np >> 3) << 17) |
                             ((uint32_t)(TC_M >> 4) << 24);
      const uint32_t sbo = (uint32_t)(Ly.Kp * 16);
      for (int ks = 0; ks < Ly.Kp / 16; ks++) {
        const uint64_t ad = smem_desc(smem_u32(A) + ks * 256, 128, sbo);
        const uint64_t bd = smem_desc(smem_u32(Bw) + ks * 256, 128, sbo);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(barM)
                   : "memory");
    }
    ok = __syncthreads_and(mbar_wait(barM, phM, err) ? 1 : 0) != 0;
    phM ^= 1u;
    if (!ok) break;
    if (tid == 0 && l + 1 < net.L) load_weights(l + 1);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const bool last = l == net.L - 1;
    const long r = row0 + rloc;
    for (int c0 = 16 * cgrp; c0 < Ly.Np; c0 += 64) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(lgrp * 32) << 16) + (uint32_t)c0)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float f[16];
#pragma unroll
      for (int q = 0; q < 16; q++) f[q] = __uint_as_float(v[q]) + (c0 + q < Ly.N ? Ly.bias[c0 + q] : 0.0f);
      if (!last) {
        __align__(16) __nv_bfloat16 h[16];
#pragma unroll
        for (int q = 0; q < 16; q++) h[q] = __float2bfloat16(c0 + q < Ly.N ? gelu_f(f[q]) : 0.0f);
        *reinterpret_cast<uint4*>(A + canon_off(rloc, c0, Ly.Np)) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(A + canon_off(rloc, c0 + 8, Ly.Np)) = *reinterpret_cast<const uint4*>(h + 8);
      } else if (r < n) {
#pragma unroll
        for (int q = 0; q < 16; q++)
          if (c0 + q < Ly.N) y[r * Ly.N + c0 + q] = f[q];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

}  // namespace

struct pic_mlp {
  std::vector<int> w;                   // widths
  int L = 0;                            // layers
  long np = 0;                          // parameters
  std::vector<long> off_w, off_b;       // offsets into the parameter vector
  float* p = nullptr;                   // FP32 master parameters
  __nv_bfloat16* pb = nullptr;          // BF16 copies
  float* g = nullptr;                   // gradient
  float* m = nullptr;
  float* v = nullptr;
  long adam_t = 0;
  int cap = 0;                          // batch capacity of the work buffers
  std::vector<float*> Z;                // pre-activations per layer (FP32)
  std::vector<__nv_bfloat16*> Hb;       // activations per layer (BF16); Hb[0] is the input
  float* dA = nullptr;                  // gradient work buffers
  float* dB = nullptr;
  float* out = nullptr;
  float* loss = nullptr;
  int* idx = nullptr;
  int* perm = nullptr;                  // shuffled sample order of one epoch (training)
  int perm_cap = 0;
  float* curve = nullptr;               // per-epoch loss sums (training)
  int curve_cap = 0;
  float2* ctab = nullptr;               // AdamW bias corrections per step of a training call
  long ctab_cap = 0;
  int* eidx = nullptr;                  // epoch index of a training call, advanced on the device
  bool use_graphs = true;               // training replays a captured epoch
  float* xb = nullptr;
  float* tb = nullptr;
  // tensor-core inference: packed weight images per layer, rebuilt when the BF16 weights change
  bool tc_ok = false;                   // every padded width <= 256
  bool tc_dirty = true;
  bool use_tc = true;
  std::vector<__nv_bfloat16*> img;
  int* err = nullptr;                   // device flag: a tensor-core wait gave up
  cudaStream_t s = nullptr;
  pic_alloc_fn alloc = nullptr;
  pic_free_fn freef = nullptr;
  void* user = nullptr;
  std::vector<std::pair<void*, size_t>> allocs;
};

namespace {

template <class X>
X* mlp_al(pic_mlp* m, size_t n) {
  const size_t b = n * sizeof(X) + 256;
  void* p = nullptr;
  if (m->alloc) p = m->alloc(b, (void*)m->s, m->user);
  else if (cudaMalloc(&p, b) != cudaSuccess) p = nullptr;
  if (p) m->allocs.emplace_back(p, b);
  return (X*)p;
}

void mlp_release(pic_mlp* m) {
  cudaStreamSynchronize(m->s);
  for (auto& a : m->allocs) {
    if (m->freef) m->freef(a.first, a.second, (void*)m->s, m->user);
    else cudaFree(a.first);
  }
  m->allocs.clear();
}

int maxw(const pic_mlp* m) {
  int r = 0;
  for (int x : m->w) r = x > r ? x : r;
  return r;
}

bool ensure_batch(pic_mlp* m, int n) {
  if (n <= m->cap) return true;
  const int wm = maxw(m);
  m->Z.assign(m->L + 1, nullptr);
  m->Hb.assign(m->L + 1, nullptr);
  for (int l = 0; l <= m->L; l++) {
    m->Z[l] = mlp_al<float>(m, (size_t)n * m->w[l]);
    m->Hb[l] = mlp_al<__nv_bfloat16>(m, (size_t)n * m->w[l]);
    if (!m->Z[l] || !m->Hb[l]) return false;
  }
  m->dA = mlp_al<float>(m, (size_t)n * wm);
  m->dB = mlp_al<float>(m, (size_t)n * wm);
  m->out = mlp_al<float>(m, (size_t)n * m->w[m->L]);
  m->xb = mlp_al<float>(m, (size_t)n * m->w[0]);
  m->tb = mlp_al<float>(m, (size_t)n * m->w[m->L]);
  m->idx = mlp_al<int>(m, (size_t)n);
  if (!m->dA || !m->dB || !m->out || !m->xb || !m->tb || !m->idx) return false;
  m->cap = n;
  return true;
}

dim3 ggrid(int M, int N) { return dim3((N + GT - 1) / GT, (M + GT - 1) / GT); }

// forward of n rows of X (FP32, n x w0) into m->out (FP32, n x wL)
void forward(pic_mlp* m, const float* X, int n) {
  const long n0 = (long)n * m->w[0];
  k_to_bf16<<<(unsigned)((n0 + 255) / 256), 256, 0, m->s>>>(n0, X, m->Hb[0]);
  for (int l = 1; l <= m->L; l++) {
    const int in = m->w[l - 1], ou = m->w[l];
    const __nv_bfloat16* W = m->pb + m->off_w[l - 1];
    const float* b = m->p + m->off_b[l - 1];
    if (l < m->L)
      k_gemm<__nv_bfloat16, __nv_bfloat16, false, true, 1><<<ggrid(n, ou), 256, 0, m->s>>>(
          n, ou, in, m->Hb[l - 1], in, W, in, m->Z[l], ou, b, m->Hb[l]);
    else
      k_gemm<__nv_bfloat16, __nv_bfloat16, false, true, 2><<<ggrid(n, ou), 256, 0, m->s>>>(
          n, ou, in, m->Hb[l - 1], in, W, in, m->out, ou, b, nullptr);
  }
}

// gradient of the mean squared error of m->out against T (n x wL) into m->g; the loss is added to *loss
void backward(pic_mlp* m, const float* T, int n, float* loss, const int* eidx = nullptr) {
  const int wl = m->w[m->L];
  const long nd = (long)n * wl;
  k_mse<<<(unsigned)((nd + 255) / 256), 256, 0, m->s>>>(nd, m->out, T, m->dA, loss, eidx);
  float* dZ = m->dA;   // gradient w.r.t. the current layer's output (pre-activation for the last)
  float* dH = m->dB;
  for (int l = m->L; l >= 1; l--) {
    const int in = m->w[l - 1], ou = m->w[l];
    // dW = dZ^T H_{l-1}: (ou x in), sum over the batch
    k_gemm<float, __nv_bfloat16, true, false, 0><<<ggrid(ou, in), 256, 0, m->s>>>(
        ou, in, n, dZ, ou, m->Hb[l - 1], in, m->g + m->off_w[l - 1], in, nullptr, nullptr);
    k_colsum<<<ou, 256, 0, m->s>>>(n, ou, dZ, m->g + m->off_b[l - 1]);
    if (l > 1) {
      // dH_{l-1} = dZ W (n x in), then through the GELU of layer l-1
      k_gemm<float, __nv_bfloat16, false, false, 0><<<ggrid(n, in), 256, 0, m->s>>>(
          n, in, ou, dZ, ou, m->pb + m->off_w[l - 1], in, dH, in, nullptr, nullptr);
      const long ne = (long)n * in;
      k_gelu_back<<<(unsigned)((ne + 255) / 256), 256, 0, m->s>>>(ne, m->Z[l - 1], dH, dH);
      float* t = dZ;
      dZ = dH;
      dH = t;
    }
  }
}

}  // namespace

extern "C" {

int pic_mlp_create(int n_layers, const int* widths, uint64_t seed, pic_alloc_fn alloc, pic_free_fn free_fn,
                   void* alloc_user, void* cuda_stream, pic_mlp** out) {
  if (!out) return PIC_EINVAL;
  *out = nullptr;
  if (n_layers < 1 || n_layers > 16 || !widths) return PIC_EINVAL;
  for (int l = 0; l <= n_layers; l++)
    if (widths[l] < 1 || widths[l] > 4096) return PIC_EINVAL;
  pic_mlp* m = new pic_mlp();
  m->L = n_layers;
  m->w.assign(widths, widths + n_layers + 1);
  m->s = (cudaStream_t)cuda_stream;
  m->alloc = alloc; m->freef = free_fn; m->user = alloc_user;
  long off = 0;
  for (int l = 1; l <= n_layers; l++) {
    m->off_w.push_back(off); off += (long)m->w[l] * m->w[l - 1];
    m->off_b.push_back(off); off += m->w[l];
  }
  m->np = off;
  m->p = mlp_al<float>(m, off);
  m->pb = mlp_al<__nv_bfloat16>(m, off);
  m->g = mlp_al<float>(m, off);
  m->m = mlp_al<float>(m, off);
  m->v = mlp_al<float>(m, off);
  m->loss = mlp_al<float>(m, 1);
  m->err = mlp_al<int>(m, 1);
  m->tc_ok = n_layers <= TC_MAXL;
  for (int l = 0; l <= n_layers; l++) m->tc_ok = m->tc_ok && pad16(widths[l]) <= TC_MAXW;
  if (m->tc_ok) {
    for (int l = 1; l <= n_layers; l++) m->img.push_back(mlp_al<__nv_bfloat16>(m, (size_t)pad16(widths[l]) * pad16(widths[l - 1])));
    for (auto* q : m->img) m->tc_ok = m->tc_ok && q;
    cudaFuncSetAttribute(k_mlp_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
  }
  if (!m->p || !m->pb || !m->g || !m->m || !m->v || !m->loss || !m->err) {
    mlp_release(m);
    delete m;
    return PIC_ENOMEM;
  }
  // He-style uniform initialisation from a counter-based generator; zero biases
  std::vector<float> h(off, 0.0f);
  uint64_t st = seed;
  for (int l = 1; l <= n_layers; l++) {
    const float a = std::sqrt(6.0f / (float)m->w[l - 1]) * (l == n_layers ? 0.5f : 1.0f);
    for (long i = 0; i < (long)m->w[l] * m->w[l - 1]; i++) {
      const double u = (double)(splitmix64(st) >> 11) * (1.0 / 9007199254740992.0);
      h[m->off_w[l - 1] + i] = (float)((2.0 * u - 1.0) * a);
    }
  }
  cudaMemcpyAsync(m->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice, m->s);
  k_to_bf16<<<(unsigned)((off + 255) / 256), 256, 0, m->s>>>(off, m->p, m->pb);
  cudaMemsetAsync(m->m, 0, off * sizeof(float), m->s);
  cudaMemsetAsync(m->v, 0, off * sizeof(float), m->s);
  cudaMemsetAsync(m->err, 0, sizeof(int), m->s);
  if (cudaStreamSynchronize(m->s) != cudaSuccess) {
    mlp_release(m);
    delete m;
    return PIC_ECUDA;
  }
  *out = m;
  return PIC_OK;
}

int pic_mlp_free(pic_mlp* m) {
  if (!m) return PIC_OK;
  mlp_release(m);
  delete m;
  return PIC_OK;
}

int64_t pic_mlp_param_count(pic_mlp* m) { return m ? m->np : 0; }

int pic_mlp_get_params(pic_mlp* m, float* dst) {
  if (!m || !dst) return PIC_EINVAL;
  return cudaMemcpyAsync(dst, m->p, m->np * sizeof(float), cudaMemcpyDeviceToHost, m->s) == cudaSuccess &&
                 cudaStreamSynchronize(m->s) == cudaSuccess
             ? PIC_OK
             : PIC_ECUDA;
}

int pic_mlp_set_params(pic_mlp* m, const float* src) {
  if (!m || !src) return PIC_EINVAL;
  cudaMemcpyAsync(m->p, src, m->np * sizeof(float), cudaMemcpyHostToDevice, m->s);
  k_to_bf16<<<(unsigned)((m->np + 255) / 256), 256, 0, m->s>>>(m->np, m->p, m->pb);
  m->adam_t = 0;
  m->tc_dirty = true;
  cudaMemsetAsync(m->m, 0, m->np * sizeof(float), m->s);
  cudaMemsetAsync(m->v, 0, m->np * sizeof(float), m->s);
  return cudaStreamSynchronize(m->s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_infer(pic_mlp* m, const float* x, int64_t n, float* y) {
  if (!m || !x || !y || n < 0) return PIC_EINVAL;
  if (n == 0) return PIC_OK;
  if (m->tc_ok && m->use_tc) {
    if (m->tc_dirty) {
      for (int l = 1; l <= m->L; l++) {
        const int N = m->w[l], K = m->w[l - 1], Np = pad16(N), Kp = pad16(K);
        k_pack_weights<<<(Np * Kp + 255) / 256, 256, 0, m->s>>>(m->pb + m->off_w[l - 1], N, K, Np, Kp, m->img[l - 1]);
      }
      m->tc_dirty = false;
    }
    TcNet net{};
    net.L = m->L;
    net.k0 = m->w[0];
    for (int l = 1; l <= m->L; l++) {
      TcLayer& t = net.l[l - 1];
      t.img = m->img[l - 1];
      t.bias = m->p + m->off_b[l - 1];
      t.N = m->w[l];
      t.K = m->w[l - 1];
      t.Np = pad16(t.N);
      t.Kp = pad16(t.K);
    }
    const long blocks = (n + TC_M - 1) / TC_M;
    k_mlp_fwd_tc<<<(unsigned)blocks, TC_THREADS, TC_SMEM, m->s>>>(net, x, (long)n, y, m->err);
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
  }
  const int chunk = 65536;
  for (int64_t r0 = 0; r0 < n; r0 += chunk) {
    const int nb = (int)(n - r0 < chunk ? n - r0 : chunk);
    if (!ensure_batch(m, nb)) return PIC_ENOMEM;
    forward(m, x + r0 * m->w[0], nb);
    cudaMemcpyAsync(y + r0 * m->w[m->L], m->out, (size_t)nb * m->w[m->L] * sizeof(float), cudaMemcpyDeviceToDevice,
                    m->s);
  }
  return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_use_tensor_cores(pic_mlp* m, int enable) {
  if (!m) return PIC_EINVAL;
  if (enable && !m->tc_ok) return PIC_EINVAL;
  m->use_tc = enable != 0;
  return PIC_OK;
}

int pic_mlp_use_graphs(pic_mlp* m, int enable) {
  if (!m) return PIC_EINVAL;
  m->use_graphs = enable != 0;
  return PIC_OK;
}

int pic_mlp_status(pic_mlp* m) {
  if (!m) return PIC_EINVAL;
  if (cudaStreamSynchronize(m->s) != cudaSuccess) return PIC_ECUDA;
  int e = 0;
  if (cudaMemcpy(&e, m->err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PIC_ECUDA;
  return e ? PIC_ETIMEOUT : PIC_OK;
}

int pic_mlp_grad(pic_mlp* m, const float* x, const float* t, int n, float* loss_host, float* grad_host) {
  if (!m || !x || !t || n < 1) return PIC_EINVAL;
  if (!ensure_batch(m, n)) return PIC_ENOMEM;
  forward(m, x, n);
  cudaMemsetAsync(m->loss, 0, sizeof(float), m->s);
  backward(m, t, n, m->loss);
  if (loss_host) cudaMemcpyAsync(loss_host, m->loss, sizeof(float), cudaMemcpyDeviceToHost, m->s);
  if (grad_host) cudaMemcpyAsync(grad_host, m->g, m->np * sizeof(float), cudaMemcpyDeviceToHost, m->s);
  return cudaStreamSynchronize(m->s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_train(pic_mlp* m, const float* x, const float* t, int n, int epochs, int batch, float lr,
                  float weight_decay, uint64_t seed, float* loss_curve) {
  if (!m || !x || !t || n < 1 || epochs < 0 || batch < 1) return PIC_EINVAL;
  if (batch > n) batch = n;
  if (!ensure_batch(m, batch)) return PIC_ENOMEM;
  if (n > m->perm_cap) {
    m->perm = mlp_al<int>(m, (size_t)n);
    if (!m->perm) return PIC_ENOMEM;
    m->perm_cap = n;
  }
  if (epochs > m->curve_cap) {
    m->curve = mlp_al<float>(m, (size_t)epochs);
    if (!m->curve) return PIC_ENOMEM;
    m->curve_cap = epochs;
  }
  if (epochs > 0) cudaMemsetAsync(m->curve, 0, (size_t)epochs * sizeof(float), m->s);
  m->tc_dirty = true;
  // the host draws every epoch's order up front (pinned by the seed), one upload per epoch
  std::vector<int> perm(n);
  uint64_t st = seed;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int nbat = n / batch;
  // AdamW's bias corrections of every step of this call, computed on the host as the per-step launches did
  const long nsteps = (long)epochs * nbat;
  std::vector<float2> ctab((size_t)(nsteps > 0 ? nsteps : 1));
  for (long q = 0; q < nsteps; q++) {
    const float tq = (float)(m->adam_t + q + 1);
    ctab[q] = make_float2(1.0f - std::pow(b1, tq), 1.0f - std::pow(b2, tq));
  }
  if (nsteps > m->ctab_cap) {
    m->ctab = mlp_al<float2>(m, (size_t)nsteps);
    if (!m->ctab) return PIC_ENOMEM;
    m->ctab_cap = nsteps;
  }
  if (!m->eidx) {
    m->eidx = mlp_al<int>(m, 1);
    if (!m->eidx) return PIC_ENOMEM;
  }
  if (nsteps > 0)
    cudaMemcpyAsync(m->ctab, ctab.data(), (size_t)nsteps * sizeof(float2), cudaMemcpyHostToDevice, m->s);
  cudaMemsetAsync(m->eidx, 0, sizeof(int), m->s);
  // one epoch's launches (nbat batches of gather, forward, backward, AdamW, then the epoch counter), with
  // the epoch index and the step's bias corrections read on the device
  auto epoch_launches = [&](cudaStream_t s) {
    cudaStream_t keep = m->s;
    m->s = s;
    for (int k = 0; k < nbat; k++) {
      k_gather_rows<<<batch, 64, 0, s>>>(batch, m->perm + (long)k * batch, x, m->w[0], t, m->w[m->L], m->xb, m->tb);
      forward(m, m->xb, batch);
      backward(m, m->tb, batch, m->curve, m->eidx);
      k_adamw<<<(unsigned)((m->np + 255) / 256), 256, 0, s>>>(m->np, m->p, m->g, m->m, m->v, m->pb, lr, b1, b2, eps,
                                                              weight_decay, 0.f, 0.f, m->ctab, m->eidx, nbat, k);
    }
    k_next_epoch<<<1, 1, 0, s>>>(m->eidx);
    m->s = keep;
  };
  // The epoch is captured once in a CUDA graph on a private stream and replayed (about 20 launches per
  // batch otherwise: at batch 64 the step is launch-bound). Where capture is not possible, the same
  // launches run directly on the caller's stream.
  cudaStream_t ts = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  if (m->use_graphs && epochs > 1 && nbat > 0 && cudaStreamIsCapturing(m->s, &cap_st) == cudaSuccess &&
      cap_st == cudaStreamCaptureStatusNone && cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking) == cudaSuccess) {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      epoch_launches(ts);
      if (cudaStreamEndCapture(ts, &gr) == cudaSuccess && gr) {
        if (cudaGraphInstantiate(&ge, gr, 0) != cudaSuccess) ge = nullptr;
        cudaGraphDestroy(gr);
      }
    }
    cudaGetLastError();   // a refused capture leaves no sticky error; the direct path follows
    if (!ge) {
      cudaStreamDestroy(ts);
      ts = nullptr;
    }
  }
  cudaEvent_t ready = nullptr;
  if (ge) {
    // the private stream starts after everything queued on the caller's stream
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventRecord(ready, m->s);
    cudaStreamWaitEvent(ts, ready, 0);
  }
  cudaStream_t run_s = ge ? ts : m->s;
  for (int e = 0; e < epochs; e++) {
    for (int i = 0; i < n; i++) perm[i] = i;
    for (int i = n - 1; i > 0; i--) {   // Fisher-Yates with a counter-based generator
      const int j = (int)(splitmix64(st) % (uint64_t)(i + 1));
      const int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    // pageable source: the copy has been staged when the call returns, so perm may be refilled
    cudaMemcpyAsync(m->perm, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, run_s);
    if (ge) cudaGraphLaunch(ge, ts);
    else epoch_launches(m->s);
  }
  m->adam_t += nsteps;
  if (ge) {
    cudaEventRecord(ready, ts);
    cudaStreamWaitEvent(m->s, ready, 0);
  }
  if (loss_curve && epochs > 0) {
    cudaMemcpyAsync(loss_curve, m->curve, (size_t)epochs * sizeof(float), cudaMemcpyDeviceToHost, m->s);
  }
  const bool ok = cudaStreamSynchronize(m->s) == cudaSuccess;
  if (ge) {
    cudaGraphExecDestroy(ge);
    cudaStreamDestroy(ts);
    cudaEventDestroy(ready);
  }
  if (!ok) return PIC_ECUDA;
  if (loss_curve)
    for (int e = 0; e < epochs; e++) loss_curve[e] /= (float)(nbat > 0 ? nbat : 1);
  return PIC_OK;
}

}  // extern "C"
