// Learned warm start: a 3-layer MLP (ReLU hidden layers, linear output)
// trained and evaluated by this library's own kernels.
//
//   h1 = relu(x W1^T + b1),  h2 = relu(h1 W2^T + b2),  y = h2 W3^T + b3
//   L  = 1/(2B) sum_b |y_b - t_b|^2,  Adam (beta1 0.9, beta2 0.999, eps 1e-8)
//
// Weights are kept as FP32 master copies (for Adam) and as BF16 copies that
// the matrix products read (row-major and, for the backward products,
// transposed); every product runs on the tensor cores (umma.cu: tcgen05 with
// TMA-staged bf16 operands and FP32 accumulation in tensor memory).
// Activations and back-propagated errors are kept in FP32 and, as the
// operands of the next products, rounded to BF16 by the product that forms
// them (row-major and transposed copies).
#include "mls_internal.cuh"

#include <algorithm>
#include <cstring>
#include <new>

namespace mls {

// dY = (Y - That) / B with That = (T - tmu) * tisd (standardised targets, when
// tmu is given; cols = width of a row), loss partials; dY is also written
// rounded to bf16, row-major [B][ld16] and transposed [cols][ld16t]
__global__ void k_mlp_dy(int n, int cols, float invB, const float* __restrict__ Y, const float* __restrict__ T,
                         const float* __restrict__ tmu, const float* __restrict__ tisd, float* __restrict__ dY,
                         __nv_bfloat16* __restrict__ dy16, int ld16, __nv_bfloat16* __restrict__ dy16t, int ld16t,
                         double* __restrict__ loss) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double l = 0.0;
  if (i < n) {
    const int r = i / cols, c = i % cols;
    const float t = tmu ? (T[i] - tmu[c]) * tisd[c] : T[i];
    const float d = Y[i] - t;
    const float g = d * invB;
    dY[i] = g;
    const __nv_bfloat16 gb = __float2bfloat16(g);
    dy16[(int64_t)r * ld16 + c] = gb;
    dy16t[(int64_t)c * ld16t + r] = gb;
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

// Adam on a flat parameter array
__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float c1, float c2, float eps) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
}

// rows order[0..B) of X [n][cols] -> out [B][cols]
__global__ void k_gather_rows(int B, int cols, const int* __restrict__ order, const float* __restrict__ X,
                              float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)B * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  out[i] = X[(int64_t)order[r] * cols + c];
}

// bf16 copy of a row-major FP32 matrix [rows][cols] with row pitch ld (dst,
// nullable) and of its transpose [cols][ldt] (dst_t, nullable); with mu the
// columns are standardised first, (a - mu[c]) isd[c]
__global__ void k_to_bf16_2d(int rows, int cols, const float* __restrict__ a, const float* __restrict__ mu,
                             const float* __restrict__ isd, __nv_bfloat16* __restrict__ dst, int ld,
                             __nv_bfloat16* __restrict__ dst_t, int ldt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * cols) return;
  const int r = (int)(i / cols), c = (int)(i % cols);
  float v = a[i];
  if (mu) v = (v - mu[c]) * isd[c];
  const __nv_bfloat16 b = __float2bfloat16(v);
  if (dst) dst[(int64_t)r * ld + c] = b;
  if (dst_t) dst_t[(int64_t)c * ldt + r] = b;
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
  int in_p = 0, hid_p = 0, out_p = 0, bat_p = 0;  // row pitches of the bf16 operands (multiples of 8)
  float* w = nullptr;            // FP32 master parameters
  // BF16 copies read by the products: W1 [hid][in_p], W2 [hid][hid_p],
  // W3 [out][hid_p], W2^T [hid][hid_p], W3^T [hid][out_p]
  __nv_bfloat16 *w1b = nullptr, *w2b = nullptr, *w3b = nullptr, *w2tb = nullptr, *w3tb = nullptr;
  // bf16 operands: (standardised) input, hidden activations and errors,
  // row-major [B][.] and transposed [.][bat_p]
  __nv_bfloat16 *xs16 = nullptr, *xs16t = nullptr, *z1_16 = nullptr, *z1_16t = nullptr, *z2_16 = nullptr,
                *z2_16t = nullptr, *dy16 = nullptr, *dy16t = nullptr, *d2_16 = nullptr, *d2_16t = nullptr,
                *d1_16t = nullptr;
  int* err = nullptr;            // set by a product whose bounded wait gave up
  float* grad = nullptr;
  float* m = nullptr;
  float* v = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *d2 = nullptr, *d1 = nullptr;
  float* tb = nullptr;                  // gathered minibatch targets
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

static inline int pad8(int v) { return (v + 7) & ~7; }

// the BF16 copies of the weights (and of W2^T, W3^T) from the FP32 masters
static void mlp_refresh_bf16(mls_mlp* p) {
  const MlpLayout& L = p->L;
  cudaStream_t s = p->stream;
  auto conv = [&](int rows, int cols, const float* a, __nv_bfloat16* d, int ld, __nv_bfloat16* dt, int ldt) {
    const int64_t n = (int64_t)rows * cols;
    k_to_bf16_2d<<<(int)((n + 255) / 256), 256, 0, s>>>(rows, cols, a, nullptr, nullptr, d, ld, dt, ldt);
  };
  conv(p->hid, p->in, p->w + L.w1, p->w1b, p->in_p, nullptr, 0);
  conv(p->hid, p->hid, p->w + L.w2, p->w2b, p->hid_p, p->w2tb, p->hid_p);
  conv(p->out, p->hid, p->w + L.w3, p->w3b, p->hid_p, p->w3tb, p->out_p);
}

static void gemm(mls_mlp* p, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                 float* C, int ldc, const GemmEpilogue& ep) {
  gemm_bf16_tn(p->stream, M, N, K, A, lda, B, ldb, C, ldc, ep, p->err);
}

// forward pass for B rows of X (float [B][in]); leaves z1, z2 (post-ReLU) and y
// (standardised outputs, or raw outputs when raw_out is set and the network
// carries a standardisation), and the bf16 operands of the next products;
// with `train` also the transposed copies the weight gradients read
static void mlp_forward(mls_mlp* p, const float* X, int B, bool raw_out = false, bool train = false) {
  const MlpLayout& L = p->L;
  cudaStream_t s = p->stream;
  const bool nrm = p->normalised;
  const int64_t nx = (int64_t)B * p->in;
  k_to_bf16_2d<<<(int)((nx + 255) / 256), 256, 0, s>>>(B, p->in, X, nrm ? p->mu_in : nullptr,
                                                      nrm ? p->isd_in : nullptr, p->xs16, p->in_p,
                                                      train ? p->xs16t : nullptr, p->bat_p);
  GemmEpilogue e1;
  e1.bias = p->w + L.b1; e1.relu = 1;
  e1.out16 = p->z1_16; e1.ld16 = p->hid_p;
  if (train) { e1.out16t = p->z1_16t; e1.ld16t = p->bat_p; }
  gemm(p, B, p->hid, p->in, p->xs16, p->in_p, p->w1b, p->in_p, p->z1, p->hid, e1);
  GemmEpilogue e2;
  e2.bias = p->w + L.b2; e2.relu = 1;
  e2.out16 = p->z2_16; e2.ld16 = p->hid_p;
  if (train) { e2.out16t = p->z2_16t; e2.ld16t = p->bat_p; }
  gemm(p, B, p->hid, p->hid, p->z1_16, p->hid_p, p->w2b, p->hid_p, p->z2, p->hid, e2);
  GemmEpilogue e3;
  e3.bias = p->w + L.b3;
  if (raw_out && nrm) { e3.oscale = p->sd_out; e3.oshift = p->mu_out; }
  gemm(p, B, p->out, p->hid, p->z2_16, p->hid_p, p->w3b, p->hid_p, p->y, p->out, e3);
}

// gradients of the loss for targets T into p->grad after a training forward
// pass on the same rows; loss accumulated in p->loss
static void mlp_backward(mls_mlp* p, const float* T, int B) {
  const MlpLayout& L = p->L;
  cudaStream_t s = p->stream;
  const int no = B * p->out;
  const bool nrm = p->normalised;
  k_mlp_dy<<<(no + 255) / 256, 256, 0, s>>>(no, p->out, 1.f / B, p->y, T, nrm ? p->mu_out : nullptr,
                                            nrm ? p->isd_out : nullptr, p->dy, p->dy16, p->out_p, p->dy16t, p->bat_p,
                                            p->loss);
  // layer 3: dW3 = dY^T h2, db3 = colsum dY, d2 = (dY W3) * [h2 > 0]
  gemm(p, p->out, p->hid, B, p->dy16t, p->bat_p, p->z2_16t, p->bat_p, p->grad + L.w3, p->hid, GemmEpilogue{});
  k_colsum<<<(p->out + 127) / 128, 128, 0, s>>>(B, p->out, p->dy, p->grad + L.b3);
  GemmEpilogue e2;
  e2.mask = p->z2;
  e2.out16 = p->d2_16; e2.ld16 = p->hid_p;
  e2.out16t = p->d2_16t; e2.ld16t = p->bat_p;
  gemm(p, B, p->hid, p->out, p->dy16, p->out_p, p->w3tb, p->out_p, p->d2, p->hid, e2);
  // layer 2
  gemm(p, p->hid, p->hid, B, p->d2_16t, p->bat_p, p->z1_16t, p->bat_p, p->grad + L.w2, p->hid, GemmEpilogue{});
  k_colsum<<<(p->hid + 127) / 128, 128, 0, s>>>(B, p->hid, p->d2, p->grad + L.b2);
  GemmEpilogue e1;
  e1.mask = p->z1;
  e1.out16t = p->d1_16t; e1.ld16t = p->bat_p;
  gemm(p, B, p->hid, p->hid, p->d2_16, p->hid_p, p->w2tb, p->hid_p, p->d1, p->hid, e1);
  // layer 1, against the (standardised) input the forward pass used
  gemm(p, p->hid, p->in, B, p->d1_16t, p->bat_p, p->xs16t, p->bat_p, p->grad + L.w1, p->in, GemmEpilogue{});
  k_colsum<<<(p->hid + 127) / 128, 128, 0, s>>>(B, p->hid, p->d1, p->grad + L.b1);
}

// the error flag of the products: cleared, and read after a synchronisation
static mls_status mlp_check(mls_mlp* p) {
  int h = 0;
  if (cudaMemcpyAsync(&h, p->err, sizeof(int), cudaMemcpyDeviceToHost, p->stream) != cudaSuccess ||
      cudaStreamSynchronize(p->stream) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  if (h) {
    cudaMemsetAsync(p->err, 0, sizeof(int), p->stream);
    return MLS_ETIMEOUT;
  }
  return MLS_OK;
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
  p->in_p = pad8(n_in); p->hid_p = pad8(n_hidden); p->out_p = pad8(n_out); p->bat_p = pad8(max_batch);
  const int64_t P = p->L.total;
  const int64_t act = (int64_t)max_batch * std::max(n_hidden, n_out);
  const size_t bat = (size_t)p->bat_p, mb = (size_t)max_batch;
  bool ok = mlp_alloc(p, (void**)&p->w, 4 * P) &&
            mlp_alloc(p, (void**)&p->w1b, 2 * (size_t)n_hidden * p->in_p) &&
            mlp_alloc(p, (void**)&p->w2b, 2 * (size_t)n_hidden * p->hid_p) &&
            mlp_alloc(p, (void**)&p->w3b, 2 * (size_t)n_out * p->hid_p) &&
            mlp_alloc(p, (void**)&p->w2tb, 2 * (size_t)n_hidden * p->hid_p) &&
            mlp_alloc(p, (void**)&p->w3tb, 2 * (size_t)n_hidden * p->out_p) &&
            mlp_alloc(p, (void**)&p->xs16, 2 * mb * p->in_p) && mlp_alloc(p, (void**)&p->xs16t, 2 * (size_t)n_in * bat) &&
            mlp_alloc(p, (void**)&p->z1_16, 2 * mb * p->hid_p) && mlp_alloc(p, (void**)&p->z1_16t, 2 * (size_t)n_hidden * bat) &&
            mlp_alloc(p, (void**)&p->z2_16, 2 * mb * p->hid_p) && mlp_alloc(p, (void**)&p->z2_16t, 2 * (size_t)n_hidden * bat) &&
            mlp_alloc(p, (void**)&p->dy16, 2 * mb * p->out_p) && mlp_alloc(p, (void**)&p->dy16t, 2 * (size_t)n_out * bat) &&
            mlp_alloc(p, (void**)&p->d2_16, 2 * mb * p->hid_p) && mlp_alloc(p, (void**)&p->d2_16t, 2 * (size_t)n_hidden * bat) &&
            mlp_alloc(p, (void**)&p->d1_16t, 2 * (size_t)n_hidden * bat) && mlp_alloc(p, (void**)&p->err, sizeof(int)) &&
            mlp_alloc(p, (void**)&p->grad, 4 * P) && mlp_alloc(p, (void**)&p->m, 4 * P) &&
            mlp_alloc(p, (void**)&p->v, 4 * P) && mlp_alloc(p, (void**)&p->z1, 4 * act) &&
            mlp_alloc(p, (void**)&p->z2, 4 * act) && mlp_alloc(p, (void**)&p->y, 4 * act) &&
            mlp_alloc(p, (void**)&p->dy, 4 * act) && mlp_alloc(p, (void**)&p->d2, 4 * act) &&
            mlp_alloc(p, (void**)&p->d1, 4 * act) && mlp_alloc(p, (void**)&p->loss, 8) &&
            mlp_alloc(p, (void**)&p->tb, 4 * (size_t)max_batch * n_out) &&
            mlp_alloc(p, (void**)&p->xg, 4 * (size_t)max_batch * n_in) &&
            mlp_alloc(p, (void**)&p->mu_in, 4 * (size_t)n_in) && mlp_alloc(p, (void**)&p->isd_in, 4 * (size_t)n_in) &&
            mlp_alloc(p, (void**)&p->mu_out, 4 * (size_t)n_out) &&
            mlp_alloc(p, (void**)&p->isd_out, 4 * (size_t)n_out) && mlp_alloc(p, (void**)&p->sd_out, 4 * (size_t)n_out);
  if (ok && cudaMallocHost((void**)&p->loss_host, 8) != cudaSuccess) { cudaGetLastError(); ok = false; }
  if (!ok) { mlp_free(p); return MLS_ENOMEM; }
  if (cudaMemcpy(p->w, init_params, 4 * P, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(p->m, 0, 4 * P) != cudaSuccess || cudaMemset(p->v, 0, 4 * P) != cudaSuccess ||
      cudaMemset(p->err, 0, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    mlp_free(p);
    return MLS_ECUDA;
  }
  mlp_refresh_bf16(p);
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
  mlp_forward(p, X, batch, true, false);
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
    mlp_forward(p, X + (int64_t)b0 * p->in, B, true, false);
    if (cudaMemcpyAsync(Y + (int64_t)b0 * p->out, p->y, 4 * (size_t)B * p->out, cudaMemcpyDeviceToDevice,
                        p->stream) != cudaSuccess) {
      cudaGetLastError();
      return MLS_ECUDA;
    }
  }
  if (cudaGetLastError() != cudaSuccess) return MLS_ECUDA;
  return mlp_check(p);
}

mls_status mls_mlp_gradients(mls_mlp* p, const float* X, const float* T, int32_t batch, float* grad_out,
                             double* loss_out) {
  if (!p || !X || !T || batch < 1 || batch > p->max_batch) return MLS_EINVAL;
  cudaMemsetAsync(p->loss, 0, 8, p->stream);
  mlp_forward(p, X, batch, false, true);
  mlp_backward(p, T, batch);
  if (grad_out) cudaMemcpyAsync(grad_out, p->grad, 4 * (size_t)p->L.total, cudaMemcpyDeviceToDevice, p->stream);
  cudaMemcpyAsync(p->loss_host, p->loss, 8, cudaMemcpyDeviceToHost, p->stream);
  if (cudaGetLastError() != cudaSuccess) return MLS_ECUDA;
  const mls_status st = mlp_check(p);
  if (st != MLS_OK) return st;
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
    mlp_forward(p, p->xg, batch, false, true);
    mlp_backward(p, p->tb, batch);
    ++p->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
    k_adam<<<(int)((p->L.total + 255) / 256), 256, 0, s>>>(p->L.total, p->w, p->grad, p->m, p->v, lr, b1, b2, c1,
                                                          c2, 1e-8f);
    mlp_refresh_bf16(p);
    ++nsteps;
  }
  cudaMemcpyAsync(p->loss_host, p->loss, 8, cudaMemcpyDeviceToHost, s);
  if (cudaGetLastError() != cudaSuccess) return MLS_ECUDA;
  const mls_status st = mlp_check(p);
  if (st != MLS_OK) return st;
  if (loss_out) *loss_out = nsteps ? *p->loss_host / nsteps : 0.0;
  return MLS_OK;
}

mls_status mls_mlp_adam_step(mls_mlp* p, const float* grad, float lr) {
  if (!p || !grad) return MLS_EINVAL;
  cudaMemcpyAsync(p->grad, grad, 4 * (size_t)p->L.total, cudaMemcpyDeviceToDevice, p->stream);
  ++p->step;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)p->step), c2 = 1.f - powf(b2, (float)p->step);
  k_adam<<<(int)((p->L.total + 255) / 256), 256, 0, p->stream>>>(p->L.total, p->w, p->grad, p->m, p->v, lr, b1, b2,
                                                                c1, c2, 1e-8f);
  mlp_refresh_bf16(p);
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
