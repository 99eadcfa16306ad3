// Learned warm start: a 3-layer MLP (ReLU hidden layers, linear output)
// trained and evaluated by this library's own kernels.
//
//   h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3
//   L  = 1/(2B) sum_b |y_b - t_b|^2,  Adam (beta1 0.9, beta2 0.999, eps 1e-8)
//
// Weights are kept as FP32 master copies (for Adam) and as BF16 copies that
// the matrix products read; products run on the tensor cores with BF16
// operands and FP32 accumulation (mma.sync m16n8k16), activations and
// gradients are FP32 in memory and rounded to BF16 when staged as operands.
#include "mls_internal.cuh"

#include <algorithm>
#include <cstring>
#include <new>

namespace mls {

// ---- generic tensor-core GEMM: C[M x N] = A[M x K] B[K x N] ---------------------------
// Element (m, k) of A is A[m * sam + k * sak] and (k, n) of B is B[k * sbk + n * sbn],
// so any transposition is a choice of strides.  Epilogue:
//   C[m * ldc + n] = acc (+ bias[n]) (then relu) (then * (mask[m * ldc + n] > 0))
//                    (then * oscale[n] + oshift[n])
// and A's elements may be standardised on load: (A - amu[k]) * aisd[k].
constexpr int GBM = 64, GBN = 64, GBK = 32;

template <typename T> __device__ __forceinline__ __nv_bfloat16 to_bf16(T v);
template <> __device__ __forceinline__ __nv_bfloat16 to_bf16<float>(float v) { return __float2bfloat16(v); }
template <> __device__ __forceinline__ __nv_bfloat16 to_bf16<__nv_bfloat16>(__nv_bfloat16 v) { return v; }

__device__ __forceinline__ uint32_t pack2(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(128) k_gemm_bf16(int M, int N, int K, const TA* __restrict__ A, int64_t sam,
                                                   int64_t sak, const TB* __restrict__ B, int64_t sbk, int64_t sbn,
                                                   float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                   int relu, const float* __restrict__ mask,
                                                   const float* __restrict__ amu, const float* __restrict__ aisd,
                                                   const float* __restrict__ oscale, const float* __restrict__ oshift) {
  __shared__ __align__(16) __nv_bfloat16 As[GBM][GBK + 8];
  __shared__ __align__(16) __nv_bfloat16 Bs[GBN][GBK + 8];  // stored [n][k]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
  const int m0 = blockIdx.y * GBM, n0 = blockIdx.x * GBN;
  const int g = lane >> 2, tq = lane & 3;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GBK) {
    for (int idx = tid; idx < GBM * GBK; idx += 128) {
      const int mm = idx / GBK, kk = idx % GBK;
      const int gm = m0 + mm, gk = k0 + kk;
      if (gm < M && gk < K) {
        if (amu) As[mm][kk] = __float2bfloat16(((float)A[gm * sam + gk * sak] - amu[gk]) * aisd[gk]);
        else As[mm][kk] = to_bf16<TA>(A[gm * sam + gk * sak]);
      } else {
        As[mm][kk] = __float2bfloat16(0.f);
      }
    }
    for (int idx = tid; idx < GBN * GBK; idx += 128) {
      const int nn = idx / GBK, kk = idx % GBK;
      const int gn = n0 + nn, gk = k0 + kk;
      Bs[nn][kk] = (gn < N && gk < K) ? to_bf16<TB>(B[gk * sbk + gn * sbn]) : __float2bfloat16(0.f);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GBK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const int r = wm + 16 * i + g;
        a[i][0] = pack2(&As[r][ks + 2 * tq]);
        a[i][1] = pack2(&As[r + 8][ks + 2 * tq]);
        a[i][2] = pack2(&As[r][ks + 2 * tq + 8]);
        a[i][3] = pack2(&As[r + 8][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int c = wn + 8 * j + g;
        b[j][0] = pack2(&Bs[c][ks + 2 * tq]);
        b[j][1] = pack2(&Bs[c][ks + 2 * tq + 8]);
      }
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
              "{%0,%1,%2,%3};\n"
              : "+f"(acc[i][j][0]), "+f"(acc[i][j][1]), "+f"(acc[i][j][2]), "+f"(acc[i][j][3])
              : "r"(a[i][0]), "r"(a[i][1]), "r"(a[i][2]), "r"(a[i][3]), "r"(b[j][0]), "r"(b[j][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int m = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0);
        const int n = n0 + wn + 8 * j + 2 * tq + (q & 1);
        if (m < M && n < N) {
          float v = acc[i][j][q];
          if (bias) v += bias[n];
          if (relu) v = fmaxf(v, 0.f);
          if (mask && !(mask[(int64_t)m * ldc + n] > 0.f)) v = 0.f;
          if (oscale) v = v * oscale[n] + oshift[n];
          C[(int64_t)m * ldc + n] = v;
        }
      }
}

template <typename TA, typename TB>
static void gemm(cudaStream_t s, int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B,
                 int64_t sbk, int64_t sbn, float* C, int ldc, const float* bias, int relu, const float* mask,
                 const float* amu = nullptr, const float* aisd = nullptr, const float* oscale = nullptr,
                 const float* oshift = nullptr) {
  dim3 grid((N + GBN - 1) / GBN, (M + GBM - 1) / GBM);
  k_gemm_bf16<TA, TB><<<grid, 128, 0, s>>>(M, N, K, A, sam, sak, B, sbk, sbn, C, ldc, bias, relu, mask, amu, aisd,
                                          oscale, oshift);
}

// dY = (Y - That) / B with That = (T - tmu) * tisd (standardised targets, when
// tmu is given; cols = width of a row), loss partials
__global__ void k_mlp_dy(int n, int cols, float invB, const float* __restrict__ Y, const float* __restrict__ T,
                         const float* __restrict__ tmu, const float* __restrict__ tisd, float* __restrict__ dY,
                         double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    const int c = i % cols;
    const float t = tmu ? (T[i] - tmu[c]) * tisd[c] : T[i];
    const float d = Y[i] - t;
    dY[i] = d * invB;
    l = 0.5 * (double)d * d * invB;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0 && loss) atomicAdd(loss, l);
}

// column sums of a row-major [rows][cols] matrix (bias gradients)
__global__ void k_colsum(int rows, int cols, const float* __restrict__ D, float* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; ++r) s += D[(int64_t)r * cols + c];
  out[c] = s;
}

// Adam on a flat parameter array, refreshing the BF16 copy
__global__ void k_adam(int64_t n, float* __restrict__ w, __nv_bfloat16* __restrict__ wb, const float* __restrict__ g,
                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2, float c1, float c2,
                       float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  if (wb) wb[i] = __float2bfloat16(wi);
}

// rows order[0..B) of X [n][cols] -> out [B][cols]
__global__ void k_gather_rows(int B, int cols, const int* __restrict__ order, const float* __restrict__ X,
                              float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  out[i] = X[(int64_t)order[r] * cols + c];
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16(a[i]);
}

}  // namespace mls

using namespace mls;

// parameter layout in one flat FP32 array: W1 [h][in], b1 [h], W2 [h][h], b2 [h], W3 [out][h], b3 [out]
struct MlpLayout {
  int64_t w1, b1, w2, b2, w3, b3, total;
};

static MlpLayout layout(int in, int h, int out) {
  MlpLayout L;
  L.w1 = 0;
  L.b1 = L.w1 + (int64_t)h * in;
  L.w2 = L.b1 + h;
  L.b2 = L.w2 + (int64_t)h * h;
  L.w3 = L.b2 + h;
  L.b3 = L.w3 + (int64_t)out * h;
  L.total = L.b3 + out;
  return L;
}

struct mls_mlp {
  int in = 0, hid = 0, out = 0, max_batch = 0;
  cudaStream_t stream = nullptr;
  MlpLayout L{};
  float* w = nullptr;            // FP32 master parameters
  __nv_bfloat16* wb = nullptr;   // BF16 copies read by the products
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
  float *xb = nullptr, *tb = nullptr;  // gathered minibatch
  float* xg = nullptr;                  // gathered (raw) minibatch input
  // standardisation: inputs (x - mu_in) / sd_in, outputs y_raw = y sd_out + mu_out
  float *mu_in = nullptr, *isd_in = nullptr, *mu_out = nullptr, *isd_out = nullptr, *sd_out = nullptr;
  bool normalised = false;
  double* loss = nullptr;
  double* loss_host = nullptr;
  int64_t step = 0;
  std::vector<void*> allocs;
};

static void mlp_free(mls_mlp* p) {
  for (void* a : p->allocs) cudaFree(a);
  if (p->loss_host) cudaFreeHost(p->loss_host);
  delete p;
}

static bool mlp_alloc(mls_mlp* p, void** dst, size_t bytes) {
  if (cudaMalloc(dst, std::max<size_t>(bytes, 16)) != cudaSuccess) { cudaGetLastError(); return false; }
  p->allocs.push_back(*dst);
  return true;
}

// forward pass for B rows of X (float [B][in]); leaves z1, z2 (post-ReLU) and y
// (standardised outputs, or raw outputs when raw_out is set and the network
// carries a standardisation)
static void mlp_forward(mls_mlp* p, const float* X, int B, bool raw_out = false) {
  const MlpLayout& L = p->L;
  cudaStream_t s = p->stream;
  const bool nrm = p->normalised;
  gemm<float, __nv_bfloat16>(s, B, p->hid, p->in, X, p->in, 1, p->wb + L.w1, 1, p->in, p->z1, p->hid,
                             p->w + L.b1, 1, nullptr, nrm ? p->mu_in : nullptr, nrm ? p->isd_in : nullptr);
  gemm<float, __nv_bfloat16>(s, B, p->hid, p->hid, p->z1, p->hid, 1, p->wb + L.w2, 1, p->hid, p->z2, p->hid,
                             p->w + L.b2, 1, nullptr);
  gemm<float, __nv_bfloat16>(s, B, p->out, p->hid, p->z2, p->hid, 1, p->wb + L.w3, 1, p->hid, p->y, p->out,
                             p->w + L.b3, 0, nullptr, nullptr, nullptr, (raw_out && nrm) ? p->sd_out : nullptr,
                             (raw_out && nrm) ? p->mu_out : nullptr);
}

// standardised copy of the network input X [B][in] (for the first layer's
// weight gradient, which needs the same operand the forward pass used)
__global__ void k_standardise(int64_t n, int cols, const float* __restrict__ X, const float* __restrict__ mu,
                              const float* __restrict__ isd, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const int c = (int)(i % cols);
    out[i] = (X[i] - mu[c]) * isd[c];
  }
}

// gradients of the loss for targets T into p->grad; loss accumulated in p->loss
static void mlp_backward(mls_mlp* p, const float* X, const float* T, int B) {
  const MlpLayout& L = p->L;
  cudaStream_t s = p->stream;
  const int no = B * p->out;
  const bool nrm = p->normalised;
  k_mlp_dy<<<(no + 255) / 256, 256, 0, s>>>(no, p->out, 1.f / B, p->y, T, nrm ? p->mu_out : nullptr,
                                            nrm ? p->isd_out : nullptr, p->dy, p->loss);
  // layer 3: dW3 = dY^T h2, db3 = colsum dY, d2 = (dY W3) * [h2 > 0]
  gemm<float, float>(s, p->out, p->hid, B, p->dy, 1, p->out, p->z2, p->hid, 1, p->grad + L.w3, p->hid, nullptr, 0,
                     nullptr);
  k_colsum<<<(p->out + 127) / 128, 128, 0, s>>>(B, p->out, p->dy, p->grad + L.b3);
  gemm<float, __nv_bfloat16>(s, B, p->hid, p->out, p->dy, p->out, 1, p->wb + L.w3, p->hid, 1, p->d2, p->hid,
                             nullptr, 0, p->z2);
  // layer 2
  gemm<float, float>(s, p->hid, p->hid, B, p->d2, 1, p->hid, p->z1, p->hid, 1, p->grad + L.w2, p->hid, nullptr, 0,
                     nullptr);
  k_colsum<<<(p->hid + 127) / 128, 128, 0, s>>>(B, p->hid, p->d2, p->grad + L.b2);
  gemm<float, __nv_bfloat16>(s, B, p->hid, p->hid, p->d2, p->hid, 1, p->wb + L.w2, p->hid, 1, p->d1, p->hid,
                             nullptr, 0, p->z1);
  // layer 1 (against the standardised input when the network carries one)
  const float* Xop = X;
  if (nrm) {
    const int64_t nx = (int64_t)B * p->in;
    k_standardise<<<(int)((nx + 255) / 256), 256, 0, s>>>(nx, p->in, X, p->mu_in, p->isd_in, p->xb);
    Xop = p->xb;
  }
  gemm<float, float>(s, p->hid, p->in, B, p->d1, 1, p->hid, Xop, p->in, 1, p->grad + L.w1, p->in, nullptr, 0,
                     nullptr);
  k_colsum<<<(p->hid + 127) / 128, 128, 0, s>>>(B, p->hid, p->d1, p->grad + L.b1);
}

extern "C" {

mls_status mls_mlp_create(mls_mlp** out, int32_t n_in, int32_t n_hidden, int32_t n_out, int32_t max_batch,
                          const float* init_params, void* stream) {
  if (!out || n_in < 1 || n_hidden < 1 || n_out < 1 || max_batch < 1 || !init_params) return MLS_EINVAL;
  *out = nullptr;
  mls_mlp* p = new (std::nothrow) mls_mlp();
  if (!p) return MLS_ENOMEM;
  p->in = n_in; p->hid = n_hidden; p->out = n_out; p->max_batch = max_batch;
  p->stream = (cudaStream_t)stream;
  p->L = layout(n_in, n_hidden, n_out);
  const int64_t P = p->L.total;
  const int64_t act = (int64_t)max_batch * std::max(n_hidden, n_out);
  bool ok = mlp_alloc(p, (void**)&p->w, 4 * P) && mlp_alloc(p, (void**)&p->wb, 2 * P) &&
            mlp_alloc(p, (void**)&p->grad, 4 * P) && mlp_alloc(p, (void**)&p->m, 4 * P) &&
            mlp_alloc(p, (void**)&p->v, 4 * P) && mlp_alloc(p, (void**)&p->z1, 4 * act) &&
            mlp_alloc(p, (void**)&p->z2, 4 * act) && mlp_alloc(p, (void**)&p->y, 4 * act) &&
            mlp_alloc(p, (void**)&p->dy, 4 * act) && mlp_alloc(p, (void**)&p->d2, 4 * act) &&
            mlp_alloc(p, (void**)&p->d1, 4 * act) && mlp_alloc(p, (void**)&p->loss, 8) &&
            mlp_alloc(p, (void**)&p->xb, 4 * (size_t)max_batch * n_in) &&
            mlp_alloc(p, (void**)&p->tb, 4 * (size_t)max_batch * n_out) &&
            mlp_alloc(p, (void**)&p->xg, 4 * (size_t)max_batch * n_in) &&
            mlp_alloc(p, (void**)&p->mu_in, 4 * (size_t)n_in) && mlp_alloc(p, (void**)&p->isd_in, 4 * (size_t)n_in) &&
            mlp_alloc(p, (void**)&p->mu_out, 4 * (size_t)n_out) &&
            mlp_alloc(p, (void**)&p->isd_out, 4 * (size_t)n_out) && mlp_alloc(p, (void**)&p->sd_out, 4 * (size_t)n_out);
  if (ok && cudaMallocHost((void**)&p->loss_host, 8) != cudaSuccess) { cudaGetLastError(); ok = false; }
  if (!ok) { mlp_free(p); return MLS_ENOMEM; }
  if (cudaMemcpy(p->w, init_params, 4 * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p->m, 0, 4 * P) != cudaSuccess || cudaMemset(p->v, 0, 4 * P) != cudaSuccess) {
    cudaGetLastError();
    mlp_free(p);
    return MLS_ECUDA;
  }
  k_to_bf16<<<(int)((P + 255) / 256), 256, 0, p->stream>>>(P, p->w, p->wb);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    mlp_free(p);
    return MLS_ECUDA;
  }
  *out = p;
  return MLS_OK;
}

mls_status mls_mlp_destroy(mls_mlp* p) {
  if (!p) return MLS_OK;
  cudaStreamSynchronize(p->stream);
  mlp_free(p);
  return MLS_OK;
}

int64_t mls_mlp_param_count(const mls_mlp* p) { return p ? p->L.total : 0; }

}  // extern "C"

namespace mls {
// raw-space forward used by the warm start (batch rows <= max_batch)
mls_status mlp_forward_raw(mls_mlp* p, const float* X, int32_t batch, float* Y, cudaStream_t stream) {
  if (!p || batch < 1 || batch > p->max_batch) return MLS_EINVAL;
  cudaStream_t keep = p->stream;
  p->stream = stream;
  mlp_forward(p, X, batch, true);
  cudaMemcpyAsync(Y, p->y, 4 * (size_t)batch * p->out, cudaMemcpyDeviceToDevice, stream);
  p->stream = keep;
  return cudaGetLastError() == cudaSuccess ? MLS_OK : MLS_ECUDA;
}

int mlp_width_in(const mls_mlp* p) { return p->in; }
int mlp_width_out(const mls_mlp* p) { return p->out; }
}  // namespace mls

extern "C" {

mls_status mls_mlp_forward(mls_mlp* p, const float* X, int32_t batch, float* Y) {
  if (!p || !X || !Y || batch < 1) return MLS_EINVAL;
  for (int b0 = 0; b0 < batch; b0 += p->max_batch) {
    const int B = std::min(p->max_batch, batch - b0);
    mlp_forward(p, X + (int64_t)b0 * p->in, B, true);
    if (cudaMemcpyAsync(Y + (int64_t)b0 * p->out, p->y, 4 * (size_t)B * p->out, cudaMemcpyDeviceToDevice,
                        p->stream) != cudaSuccess) {
      cudaGetLastError();
      return MLS_ECUDA;
    }
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  return MLS_OK;
}

mls_status mls_mlp_gradients(mls_mlp* p, const float* X, const float* T, int32_t batch, float* grad_out,
                             double* loss_out) {
  if (!p || !X || !T || batch < 1 || batch > p->max_batch) return MLS_EINVAL;
  cudaMemsetAsync(p->loss, 0, 8, p->stream);
  mlp_forward(p, X, batch);
  mlp_backward(p, X, T, batch);
  if (grad_out) cudaMemcpyAsync(grad_out, p->grad, 4 * (size_t)p->L.total, cudaMemcpyDeviceToDevice, p->stream);
  cudaMemcpyAsync(p->loss_host, p->loss, 8, cudaMemcpyDeviceToHost, p->stream);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  if (loss_out) *loss_out = *p->loss_host;
  return MLS_OK;
}

mls_status mls_mlp_train(mls_mlp* p, const float* X, const float* T, int32_t n_samples, const int32_t* order,
                         int32_t n_order, int32_t batch, float lr, double* loss_out) {
  if (!p || !X || !T || n_samples < 1 || batch < 1 || batch > p->max_batch || !order || n_order < batch)
    return MLS_EINVAL;
  cudaStream_t s = p->stream;
  cudaMemsetAsync(p->loss, 0, 8, s);
  int nsteps = 0;
  for (int b0 = 0; b0 + batch <= n_order; b0 += batch) {
    const int64_t nx = (int64_t)batch * p->in, nt = (int64_t)batch * p->out;
    k_gather_rows<<<(int)((nx + 255) / 256), 256, 0, s>>>(batch, p->in, order + b0, X, p->xg);
    k_gather_rows<<<(int)((nt + 255) / 256), 256, 0, s>>>(batch, p->out, order + b0, T, p->tb);
    mlp_forward(p, p->xg, batch);
    mlp_backward(p, p->xg, p->tb, batch);
    ++p->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
    k_adam<<<(int)((p->L.total + 255) / 256), 256, 0, s>>>(p->L.total, p->w, p->wb, p->grad, p->m, p->v, lr, b1,
                                                          b2, c1, c2, 1e-8f);
    ++nsteps;
  }
  cudaMemcpyAsync(p->loss_host, p->loss, 8, cudaMemcpyDeviceToHost, s);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  if (loss_out) *loss_out = nsteps ? *p->loss_host / nsteps : 0.0;
  return MLS_OK;
}

mls_status mls_mlp_adam_step(mls_mlp* p, const float* grad, float lr) {
  if (!p || !grad) return MLS_EINVAL;
  cudaMemcpyAsync(p->grad, grad, 4 * (size_t)p->L.total, cudaMemcpyDeviceToDevice, p->stream);
  ++p->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
  k_adam<<<(int)((p->L.total + 255) / 256), 256, 0, p->stream>>>(p->L.total, p->w, p->wb, p->grad, p->m, p->v, lr,
                                                                b1, b2, c1, c2, 1e-8f);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  return MLS_OK;
}

__global__ void k_inv(int n, const float* __restrict__ a, float* __restrict__ b, float* __restrict__ copy) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const float v = a[i] > 0.f ? a[i] : 1.f;
    b[i] = 1.f / v;
    if (copy) copy[i] = v;
  }
}

mls_status mls_mlp_set_normalization(mls_mlp* p, const float* mean_in, const float* std_in, const float* mean_out,
                                     const float* std_out) {
  if (!p) return MLS_EINVAL;
  if (!mean_in || !std_in || !mean_out || !std_out) {
    p->normalised = false;
    return MLS_OK;
  }
  cudaStream_t s = p->stream;
  cudaMemcpyAsync(p->mu_in, mean_in, 4 * (size_t)p->in, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(p->mu_out, mean_out, 4 * (size_t)p->out, cudaMemcpyDeviceToDevice, s);
  k_inv<<<(p->in + 255) / 256, 256, 0, s>>>(p->in, std_in, p->isd_in, nullptr);
  k_inv<<<(p->out + 255) / 256, 256, 0, s>>>(p->out, std_out, p->isd_out, p->sd_out);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  p->normalised = true;
  return MLS_OK;
}

// column means and standard deviations of X [n][d] (float64 accumulation)
__global__ void k_colstats(int n, int d, const float* __restrict__ X, float* __restrict__ mean,
                           float* __restrict__ sd) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  double s = 0.0, s2 = 0.0;
  for (int r = 0; r < n; ++r) {
    const double v = X[(int64_t)r * d + c];
    s += v;
    s2 += v * v;
  }
  const double m = s / n;
  mean[c] = (float)m;
  sd[c] = (float)sqrt(fmax(s2 / n - m * m, 0.0));
}

mls_status mls_mlp_column_stats(const float* X, int32_t n, int32_t d, float* mean, float* sd, void* stream) {
  if (!X || !mean || !sd || n < 1 || d < 1) return MLS_EINVAL;
  k_colstats<<<(d + 127) / 128, 128, 0, (cudaStream_t)stream>>>(n, d, X, mean, sd);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  return MLS_OK;
}

mls_status mls_mlp_get_params(mls_mlp* p, float* host_params) {
  if (!p || !host_params) return MLS_EINVAL;
  if (cudaStreamSynchronize(p->stream) != cudaSuccess ||
      cudaMemcpy(host_params, p->w, 4 * (size_t)p->L.total, cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  return MLS_OK;
}

}  // extern "C"
