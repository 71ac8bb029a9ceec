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
__global__ void k_mse(long nd, const float* Y, const float* T, float* dY, float* loss) {
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
  if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

__global__ void k_to_bf16(long n, const float* src, __nv_bfloat16* dst) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = __float2bfloat16(src[i]);
}

// AdamW (decoupled weight decay) on the FP32 master parameters, then their BF16 copies
__global__ void k_adamw(long n, float* p, const float* g, float* m, float* v, __nv_bfloat16* pb, float lr, float b1,
                        float b2, float eps, float wd, float c1, float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
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
  float* xb = nullptr;
  float* tb = nullptr;
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
void backward(pic_mlp* m, const float* T, int n, float* loss) {
  const int wl = m->w[m->L];
  const long nd = (long)n * wl;
  k_mse<<<(unsigned)((nd + 255) / 256), 256, 0, m->s>>>(nd, m->out, T, m->dA, loss);
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
  if (!m->p || !m->pb || !m->g || !m->m || !m->v || !m->loss) {
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
  cudaMemsetAsync(m->m, 0, m->np * sizeof(float), m->s);
  cudaMemsetAsync(m->v, 0, m->np * sizeof(float), m->s);
  return cudaStreamSynchronize(m->s) == cudaSuccess ? PIC_OK : PIC_ECUDA;
}

int pic_mlp_infer(pic_mlp* m, const float* x, int64_t n, float* y) {
  if (!m || !x || !y || n < 0) return PIC_EINVAL;
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
  // the host draws every epoch's order up front (pinned by the seed), one upload per epoch
  std::vector<int> perm(n);
  uint64_t st = seed;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const int nbat = n / batch;
  for (int e = 0; e < epochs; e++) {
    for (int i = 0; i < n; i++) perm[i] = i;
    for (int i = n - 1; i > 0; i--) {   // Fisher-Yates with a counter-based generator
      const int j = (int)(splitmix64(st) % (uint64_t)(i + 1));
      const int tmp = perm[i]; perm[i] = perm[j]; perm[j] = tmp;
    }
    // pageable source: the copy has been staged when the call returns, so perm may be refilled
    cudaMemcpyAsync(m->perm, perm.data(), (size_t)n * sizeof(int), cudaMemcpyHostToDevice, m->s);
    for (int k = 0; k < nbat; k++) {
      k_gather_rows<<<batch, 64, 0, m->s>>>(batch, m->perm + (long)k * batch, x, m->w[0], t, m->w[m->L], m->xb,
                                            m->tb);
      forward(m, m->xb, batch);
      backward(m, m->tb, batch, m->curve + e);
      m->adam_t++;
      const float c1 = 1.0f - std::pow(b1, (float)m->adam_t), c2 = 1.0f - std::pow(b2, (float)m->adam_t);
      k_adamw<<<(unsigned)((m->np + 255) / 256), 256, 0, m->s>>>(m->np, m->p, m->g, m->m, m->v, m->pb, lr, b1, b2,
                                                                 eps, weight_decay, c1, c2);
    }
  }
  if (loss_curve && epochs > 0) {
    cudaMemcpyAsync(loss_curve, m->curve, (size_t)epochs * sizeof(float), cudaMemcpyDeviceToHost, m->s);
  }
  if (cudaStreamSynchronize(m->s) != cudaSuccess) return PIC_ECUDA;
  if (loss_curve)
    for (int e = 0; e < epochs; e++) loss_curve[e] /= (float)(nbat > 0 ? nbat : 1);
  return PIC_OK;
}

}  // extern "C"
