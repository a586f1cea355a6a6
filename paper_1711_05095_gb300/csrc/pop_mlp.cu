// Learned guiding potential: training of the window network on the GPU.
//
// U(C) = sum_i phi(w_i(C)) with w_i the 9 sites i-4..i+4 (bit k = site i-4+k) and phi
// an MLP 9 -> 128 -> 128 -> 1 with GELU.  It is trained as a classifier separating
// configurations of the time-averaged (ancestral) distribution p_ave (label 1) from
// the end-of-interval distribution p_end (label 0) of a biased population (Sec. 2.2,
// eqs. Opave and Opend).  For the SSEP the tilted generator is symmetric, so
// ln(p_ave / p_end) = ln v + const with v its top eigenvector, i.e. U/2 of the optimal
// control; the logit of a configuration is z = (1/2) sum_i phi(w_i) + c.
//
// A window takes only 512 values, so the network runs once per pattern (a 512-row
// batch), the logits are table look-ups, and dL/dPhi_p = (1/2) sum_n dz_n n_p(C_n).
// The two 512x128x128 products of the forward and backward passes and the 128x128x512
// weight gradient run on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32
// accumulation); the 9-input layer, the 128 -> 1 layer, the look-ups and Adam use
// FP32 CUDA cores.  Parameters (FP32 master copy) in this order: W1[128][9], b1[128],
// W2[128][128], b2[128], W3[128], b3, c.
#include <cuda_bf16.h>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>

#include "pop.h"

namespace popmlp {

constexpr int kH = POP_MLP_HIDDEN;   // 128
constexpr int kPat = 512;            // window patterns
constexpr int kNP = POP_MLP_PARAMS;  // 17922
constexpr int oW1 = 0, ob1 = oW1 + kH * 9, oW2 = ob1 + kH, ob2 = oW2 + kH * kH, oW3 = ob2 + kH,
              ob3 = oW3 + kH, oc = ob3 + 1;
static_assert(oc + 1 == kNP, "parameter layout");

struct Work {
  float* theta;  // [kNP]
  float* m;      // Adam first moment
  float* v;      // Adam second moment
  float* grad;   // [kNP]
  float* Z1;     // [512][128] pre-activations
  float* H1;
  float* Z2;
  float* H2;
  float* Phi;    // [512]
  float* dPhi;   // [512]
  float* dZ2;    // [512][128]
  float* dZ1;
  double* loss;  // sum over the batch
};

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// GELU(x) = x Phi(x) with Phi(x) = erfc(-x / sqrt 2) / 2: the complementary error
// function keeps the relative accuracy for negative x, where 1 + erf would cancel.
__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * erfcf(x * -0.70710678118654752f);
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * erfcf(x * -0.70710678118654752f) + x * expf(-0.5f * x * x) * 0.39894228040143268f;
}

// Layer 1 (9 binary inputs): Z1 = X bf16(W1)^T + b1 in FP32, b1 first and then the set
// inputs in increasing k (a fixed order, so Z1 is reproducible bit for bit), H1 = GELU(Z1).
__global__ void k_layer1(Work w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // p * 128 + h
  if (i >= kPat * kH) return;
  const int p = i / kH, h = i % kH;
  float z = w.theta[ob1 + h];
  for (int k = 0; k < 9; ++k)
    if ((p >> k) & 1) z += bf(w.theta[oW1 + h * 9 + k]);
  w.Z1[i] = z;
  w.H1[i] = gelu(z);
}

// C = A B with A(m, k) = A[m sam + k sak], B(k, n) = B[k sbk + n sbn], operands rounded
// to BF16, FP32 accumulation on the tensor cores.  One warp per 16 x 8 tile of C;
// M % 16 == 0, N % 8 == 0, K % 16 == 0.  Fragment layout of mma.m16n8k16 (PTX ISA):
// g = lane / 4, t = lane % 4; A: (g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..), (g+8, 2t+8..);
// B: (k = 2t..2t+1, n = g), (k = 2t+8.., n = g); C: (g, 2t..2t+1), (g+8, 2t..2t+1).
enum Epilogue { kStore = 0, kBiasGelu = 1, kTimesGeluGrad = 2 };

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &v, 4);
  return u;
}

template <int EPI>
__global__ void k_gemm_bf16(const float* A, int sam, int sak, const float* Bm, int sbk, int sbn,
                            int M, int N, int K, float* C, int ldc, const float* bias,
                            const float* aux, float* C2) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const int tiles_n = N / 8;
  if (warp >= (M / 16) * tiles_n) return;
  const int m0 = (warp / tiles_n) * 16, n0 = (warp % tiles_n) * 8;
  const int g = lane >> 2, t = lane & 3;
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
  auto a = [&](int m, int k) { return A[(size_t)m * sam + (size_t)k * sak]; };
  auto b = [&](int k, int n) { return Bm[(size_t)k * sbk + (size_t)n * sbn]; };
  for (int k0 = 0; k0 < K; k0 += 16) {
    const uint32_t a0 = pack_bf16(a(m0 + g, k0 + 2 * t), a(m0 + g, k0 + 2 * t + 1));
    const uint32_t a1 = pack_bf16(a(m0 + g + 8, k0 + 2 * t), a(m0 + g + 8, k0 + 2 * t + 1));
    const uint32_t a2 = pack_bf16(a(m0 + g, k0 + 2 * t + 8), a(m0 + g, k0 + 2 * t + 9));
    const uint32_t a3 = pack_bf16(a(m0 + g + 8, k0 + 2 * t + 8), a(m0 + g + 8, k0 + 2 * t + 9));
    const uint32_t b0 = pack_bf16(b(k0 + 2 * t, n0 + g), b(k0 + 2 * t + 1, n0 + g));
    const uint32_t b1 = pack_bf16(b(k0 + 2 * t + 8, n0 + g), b(k0 + 2 * t + 9, n0 + g));
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c0), "+f"(c1), "+f"(c2), "+f"(c3)
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
  }
  const int rows[2] = {m0 + g, m0 + g + 8};
  const float vals[4] = {c0, c1, c2, c3};
  for (int q = 0; q < 4; ++q) {
    const int m = rows[q >> 1], n = n0 + 2 * t + (q & 1);
    float v = vals[q];
    const size_t at = (size_t)m * ldc + n;
    if (EPI == kBiasGelu) {
      v += bias[n];
      C[at] = v;
      C2[at] = gelu(v);
    } else if (EPI == kTimesGeluGrad) {
      C[at] = v * gelu_grad(aux[at]);
    } else {
      C[at] = v;
    }
  }
}

// Layer 3: Phi_p = bf16(H2_p) . bf16(W3) + b3, one warp per pattern.
__global__ void k_layer3(Work w) {
  const int p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (p >= kPat) return;
  float s = 0.f;
  for (int h = lane; h < kH; h += 32) s += bf(w.H2[p * kH + h]) * bf(w.theta[oW3 + h]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w.Phi[p] = s + w.theta[ob3];
}

// Logits, loss and dL/dPhi of a batch: one configuration per thread.  z = (1/2)
// sum_i Phi(w_i) + c; loss softplus(z) - y z; dz = (sigmoid(z) - y) / n;
// dPhi_p += dz / 2 per window showing p; dc += dz.
__global__ void k_logits(Work w, const unsigned long long* lat, int W, int L,
                         const uint8_t* labels, int64_t n) {
  __shared__ float s_phi[kPat];
  __shared__ float s_dphi[kPat];
  __shared__ float s_dc;
  __shared__ double s_loss;
  for (int i = threadIdx.x; i < kPat; i += blockDim.x) {
    s_phi[i] = w.Phi[i];
    s_dphi[i] = 0.f;
  }
  if (threadIdx.x == 0) {
    s_dc = 0.f;
    s_loss = 0.0;
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n) {
    const unsigned long long x0 = lat[j * W], x1 = W > 1 ? lat[j * W + 1] : 0ull;
    auto site = [&](int i) -> uint32_t {
      return (uint32_t)(((i < 64 ? x0 >> i : x1 >> (i - 64))) & 1ull);
    };
    // sliding 9-bit window: pattern of window i = sites i-4 .. i+4
    uint32_t pat = 0;
    for (int k = 0; k < 9; ++k) pat |= site(((k - 4) % L + L) % L) << k;
    float acc = 0.f;
    for (int i = 0; i < L; ++i) {
      acc += s_phi[pat];
      pat = (pat >> 1) | (site((i + 5) % L) << 8);
    }
    const float z = 0.5f * acc + w.theta[oc];
    const float y = (float)labels[j];
    const float loss = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z))) - y * z;
    const float dz = (1.0f / (1.0f + expf(-z)) - y) / (float)n;
    pat = 0;
    for (int k = 0; k < 9; ++k) pat |= site(((k - 4) % L + L) % L) << k;
    for (int i = 0; i < L; ++i) {
      atomicAdd(&s_dphi[pat], 0.5f * dz);
      pat = (pat >> 1) | (site((i + 5) % L) << 8);
    }
    atomicAdd(&s_dc, dz);
    atomicAdd(&s_loss, (double)loss);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kPat; i += blockDim.x)
    if (s_dphi[i] != 0.f) atomicAdd(&w.dPhi[i], s_dphi[i]);
  if (threadIdx.x == 0) {
    atomicAdd(&w.grad[oc], s_dc);
    atomicAdd(w.loss, s_loss);
  }
}

// dW3_h = sum_p bf16(H2_ph) dPhi_p (one warp per h), db3 = sum_p dPhi_p (warp kH), and
// dZ2 = dPhi bf16(W3)^T * GELU'(Z2).
__global__ void k_back3(Work w) {
  const int wi = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wi > kH) return;
  float s = 0.f;
  for (int p = lane; p < kPat; p += 32) s += (wi < kH ? bf(w.H2[p * kH + wi]) : 1.0f) * w.dPhi[p];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) w.grad[wi < kH ? oW3 + wi : ob3] = s;
}

__global__ void k_dz2(Work w) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kPat * kH) return;
  const int p = i / kH, h = i % kH;
  w.dZ2[i] = w.dPhi[p] * bf(w.theta[oW3 + h]) * gelu_grad(w.Z2[i]);
}

// Column sums over the 512 patterns: db2 from dZ2, db1 and dW1 from dZ1 (dW1_hk =
// sum_p dZ1_ph bit_k(p)).  One warp per hidden unit.
__global__ void k_colsums(Work w) {
  const int h = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (h >= kH) return;
  float s2 = 0.f, s1 = 0.f, sk[9];
  for (int k = 0; k < 9; ++k) sk[k] = 0.f;
  for (int p = lane; p < kPat; p += 32) {
    s2 += w.dZ2[p * kH + h];
    const float d1 = w.dZ1[p * kH + h];
    s1 += d1;
    for (int k = 0; k < 9; ++k)
      if ((p >> k) & 1) sk[k] += d1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    for (int k = 0; k < 9; ++k) sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], o);
  }
  if (lane == 0) {
    w.grad[ob2 + h] = s2;
    w.grad[ob1 + h] = s1;
    for (int k = 0; k < 9; ++k) w.grad[oW1 + h * 9 + k] = sk[k];
  }
}

// Adam (Kingma & Ba) on the FP32 master parameters.
__global__ void k_adam(Work w, float lr, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kNP) return;
  const float g = w.grad[i];
  const float m = 0.9f * w.m[i] + 0.1f * g;
  const float v = 0.999f * w.v[i] + 0.001f * g * g;
  w.m[i] = m;
  w.v[i] = v;
  w.theta[i] -= lr * (m / bc1) / (sqrtf(v / bc2) + 1e-8f);
}

size_t align256(size_t x) { return (x + 255u) & ~(size_t)255u; }

struct Layout {
  size_t theta, m, v, grad, Z1, H1, Z2, H2, Phi, dPhi, dZ2, dZ1, loss, total;
};

Layout layout() {
  Layout l{};
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  l.theta = take(kNP * 4);
  l.m = take(kNP * 4);
  l.v = take(kNP * 4);
  l.grad = take(kNP * 4);
  l.Z1 = take(kPat * kH * 4);
  l.H1 = take(kPat * kH * 4);
  l.Z2 = take(kPat * kH * 4);
  l.H2 = take(kPat * kH * 4);
  l.Phi = take(kPat * 4);
  l.dPhi = take(kPat * 4);
  l.dZ2 = take(kPat * kH * 4);
  l.dZ1 = take(kPat * kH * 4);
  l.loss = take(8);
  l.total = o;
  return l;
}

}  // namespace popmlp

using namespace popmlp;

struct pop_mlp {
  Work w{};
  unsigned char* ws = nullptr;
  cudaStream_t stream = nullptr;
  int64_t steps = 0;
};

namespace {

#define MLP_CUDA(call)                             \
  do {                                             \
    if ((call) != cudaSuccess) return POP_ERR_CUDA; \
  } while (0)

int forward(pop_mlp_t* h) {
  Work& w = h->w;
  cudaStream_t st = h->stream;
  k_layer1<<<kPat * kH / 256, 256, 0, st>>>(w);
  // Z2 = bf16(H1) bf16(W2)^T + b2, H2 = GELU(Z2)
  k_gemm_bf16<kBiasGelu><<<(kPat / 16) * (kH / 8) / 4, 128, 0, st>>>(
      w.H1, kH, 1, w.theta + oW2, 1, kH, kPat, kH, kH, w.Z2, kH, w.theta + ob2, nullptr, w.H2);
  k_layer3<<<kPat * 32 / 256, 256, 0, st>>>(w);
  return cudaGetLastError() == cudaSuccess ? POP_OK : POP_ERR_CUDA;
}

int backward(pop_mlp_t* h, const uint64_t* d_lat, int32_t W, int32_t L, const uint8_t* d_lab,
             int64_t n) {
  Work& w = h->w;
  cudaStream_t st = h->stream;
  MLP_CUDA(cudaMemsetAsync(w.grad, 0, kNP * 4, st));
  MLP_CUDA(cudaMemsetAsync(w.dPhi, 0, kPat * 4, st));
  MLP_CUDA(cudaMemsetAsync(w.loss, 0, 8, st));
  k_logits<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(w, (const unsigned long long*)d_lat, W, L,
                                                        d_lab, n);
  k_back3<<<(kH + 1 + 7) / 8, 256, 0, st>>>(w);
  k_dz2<<<kPat * kH / 256, 256, 0, st>>>(w);
  // dW2 = bf16(dZ2)^T bf16(H1): M = 128 (out), N = 128 (in), K = 512
  k_gemm_bf16<kStore><<<(kH / 16) * (kH / 8) / 4, 128, 0, st>>>(
      w.dZ2, 1, kH, w.H1, kH, 1, kH, kH, kPat, w.grad + oW2, kH, nullptr, nullptr, nullptr);
  // dZ1 = (bf16(dZ2) bf16(W2)) * GELU'(Z1): M = 512, N = 128, K = 128
  k_gemm_bf16<kTimesGeluGrad><<<(kPat / 16) * (kH / 8) / 4, 128, 0, st>>>(
      w.dZ2, kH, 1, w.theta + oW2, kH, 1, kPat, kH, kH, w.dZ1, kH, nullptr, w.Z1, nullptr);
  k_colsums<<<kH * 32 / 256, 256, 0, st>>>(w);
  return cudaGetLastError() == cudaSuccess ? POP_OK : POP_ERR_CUDA;
}

bool valid_batch(const uint64_t* d_lat, int32_t W, int32_t L, const uint8_t* d_lab, int64_t n) {
  return d_lat != nullptr && d_lab != nullptr && n >= 1 && n <= (1ll << 30) && W >= 1 && W <= 2 &&
         L >= 9 && L <= 64 * W;
}

}  // namespace

extern "C" {

size_t pop_mlp_workspace_bytes(void) { return layout().total; }

int pop_mlp_init(pop_mlp_t** out, const float* h_theta, void* d_workspace, size_t workspace_bytes,
                 void* cuda_stream) {
  if (out == nullptr) return POP_ERR_ARG;
  *out = nullptr;
  const Layout l = layout();
  if (h_theta == nullptr || d_workspace == nullptr || workspace_bytes < l.total ||
      ((uintptr_t)d_workspace & 255u) != 0)
    return POP_ERR_ARG;
  pop_mlp_t* h = new (std::nothrow) pop_mlp();
  if (h == nullptr) return POP_ERR_ARG;
  h->ws = (unsigned char*)d_workspace;
  h->stream = (cudaStream_t)cuda_stream;
  Work& w = h->w;
  w.theta = (float*)(h->ws + l.theta);
  w.m = (float*)(h->ws + l.m);
  w.v = (float*)(h->ws + l.v);
  w.grad = (float*)(h->ws + l.grad);
  w.Z1 = (float*)(h->ws + l.Z1);
  w.H1 = (float*)(h->ws + l.H1);
  w.Z2 = (float*)(h->ws + l.Z2);
  w.H2 = (float*)(h->ws + l.H2);
  w.Phi = (float*)(h->ws + l.Phi);
  w.dPhi = (float*)(h->ws + l.dPhi);
  w.dZ2 = (float*)(h->ws + l.dZ2);
  w.dZ1 = (float*)(h->ws + l.dZ1);
  w.loss = (double*)(h->ws + l.loss);
  if (cudaMemsetAsync(h->ws, 0, l.total, h->stream) != cudaSuccess ||
      cudaMemcpyAsync(w.theta, h_theta, kNP * 4, cudaMemcpyHostToDevice, h->stream) != cudaSuccess ||
      cudaStreamSynchronize(h->stream) != cudaSuccess) {
    delete h;
    return POP_ERR_CUDA;
  }
  *out = h;
  return POP_OK;
}

int pop_mlp_grad(pop_mlp_t* h, const uint64_t* d_lattice, int32_t W, int32_t L,
                 const uint8_t* d_labels, int64_t n, double* h_loss, float* h_grad) {
  if (h == nullptr || !valid_batch(d_lattice, W, L, d_labels, n)) return POP_ERR_ARG;
  int rc = forward(h);
  if (rc == POP_OK) rc = backward(h, d_lattice, W, L, d_labels, n);
  if (rc != POP_OK) return rc;
  double loss = 0.0;
  MLP_CUDA(cudaMemcpyAsync(&loss, h->w.loss, 8, cudaMemcpyDeviceToHost, h->stream));
  if (h_grad) MLP_CUDA(cudaMemcpyAsync(h_grad, h->w.grad, kNP * 4, cudaMemcpyDeviceToHost, h->stream));
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  if (h_loss) *h_loss = loss / (double)n;
  return POP_OK;
}

int pop_mlp_step(pop_mlp_t* h, const uint64_t* d_lattice, int32_t W, int32_t L,
                 const uint8_t* d_labels, int64_t n, float lr, double* h_loss) {
  if (h == nullptr || !valid_batch(d_lattice, W, L, d_labels, n) || !(lr > 0.0f)) return POP_ERR_ARG;
  int rc = forward(h);
  if (rc == POP_OK) rc = backward(h, d_lattice, W, L, d_labels, n);
  if (rc != POP_OK) return rc;
  h->steps += 1;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)h->steps));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)h->steps));
  k_adam<<<(kNP + 255) / 256, 256, 0, h->stream>>>(h->w, lr, bc1, bc2);
  MLP_CUDA(cudaGetLastError());
  if (h_loss) {
    double loss = 0.0;
    MLP_CUDA(cudaMemcpyAsync(&loss, h->w.loss, 8, cudaMemcpyDeviceToHost, h->stream));
    MLP_CUDA(cudaStreamSynchronize(h->stream));
    *h_loss = loss / (double)n;
  }
  return POP_OK;
}

int pop_mlp_params(pop_mlp_t* h, float* h_theta) {
  if (h == nullptr || h_theta == nullptr) return POP_ERR_ARG;
  MLP_CUDA(cudaMemcpyAsync(h_theta, h->w.theta, kNP * 4, cudaMemcpyDeviceToHost, h->stream));
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  return POP_OK;
}

int pop_mlp_potential(pop_mlp_t* h, float* h_phi) {
  if (h == nullptr || h_phi == nullptr) return POP_ERR_ARG;
  const int rc = forward(h);
  if (rc != POP_OK) return rc;
  MLP_CUDA(cudaMemcpyAsync(h_phi, h->w.Phi, kPat * 4, cudaMemcpyDeviceToHost, h->stream));
  MLP_CUDA(cudaStreamSynchronize(h->stream));
  return POP_OK;
}

void pop_mlp_free(pop_mlp_t* h) { delete h; }

}  // extern "C"
