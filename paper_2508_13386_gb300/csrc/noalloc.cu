// Allocation-free variant of the elastic energy reduction.
//
// Some callers cannot call cudaMalloc while they run: code that executes
// between pre-planned allocations (a real-time loop with a fixed memory
// budget, a host framework that owns every device allocation, or work issued
// where allocating would synchronise the device).  This entry point needs no
// context and allocates nothing: its grid-reduction scratch is a file-scope
// __device__ array, and all inputs and outputs are buffers the caller
// already owns.
//
// Limits and sharing:
//  * at most kNoallocMaxBlocks blocks of kNoallocThreads threads, i.e.
//    MLS_NOALLOC_MAX_TETS tets per call; larger meshes are rejected;
//  * the scratch lives as long as the library is loaded, on every device
//    that has called the entry point (about 48 KB each);
//  * every call shares it: the completion counter is cleared at the start of
//    each call, and two calls whose kernels overlap on the GPU (different
//    streams, or different host threads on one device) race on it and give
//    wrong results; serialise them;
//  * the first call on a device looks up the scratch's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture.  The address belongs to the device's
//    primary context and is cached for the life of the process, so a
//    caller that resets the device (cudaDeviceReset) must not call this
//    entry point on it afterwards.
#include "mls_internal.cuh"

#include <mutex>

namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocMaxBlocks = 4096;
constexpr int kNoallocMaxDevices = 64;

struct NoallocScratch {
  double partial[kNoallocMaxBlocks];
  int invalid[kNoallocMaxBlocks];
  unsigned int counter;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// device address of g_noalloc_scratch per device, looked up once
NoallocScratch* g_scratch_ptr[kNoallocMaxDevices] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ double det3_na(const double (&A)[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// one thread per tet: vol psi(F) with the rest shape formed from X; tets with
// an index outside [0, n), a non-positive rest volume or J <= 0 contribute no
// energy and are counted as invalid
__global__ void __launch_bounds__(kNoallocThreads) k_elastic_energy_noalloc(
    int n, int t, const double* __restrict__ X, const int* __restrict__ tets, const double* __restrict__ mu,
    const double* __restrict__ lam, const double* __restrict__ x, NoallocScratch* __restrict__ s,
    double* __restrict__ energy_out, int* __restrict__ invalid_out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  double en = 0.0;
  int bad = 0;
  if (e < t) {
    int v[4];
    bool ok = true;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      v[a] = tets[4 * e + a];
      ok = ok && v[a] >= 0 && v[a] < n;
    }
    if (ok) {
      double Dm[3][3], Ds[3][3];
#pragma unroll
      for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          Dm[c][k] = X[3 * v[k + 1] + c] - X[3 * v[0] + c];
          Ds[c][k] = x[3 * v[k + 1] + c] - x[3 * v[0] + c];
        }
      const double dm = det3_na(Dm);
      const double ds = det3_na(Ds);
      if (dm > 0.0 && ds > 0.0) {
        // F = Ds Dm^{-1};  |F|^2 from Ds cof(Dm)^T / det(Dm);  J = det Ds / det Dm
        double C[3][3];  // cofactor matrix of Dm: Dm^{-1} = C^T / dm
        C[0][0] = Dm[1][1] * Dm[2][2] - Dm[1][2] * Dm[2][1];
        C[0][1] = Dm[1][2] * Dm[2][0] - Dm[1][0] * Dm[2][2];
        C[0][2] = Dm[1][0] * Dm[2][1] - Dm[1][1] * Dm[2][0];
        C[1][0] = Dm[0][2] * Dm[2][1] - Dm[0][1] * Dm[2][2];
        C[1][1] = Dm[0][0] * Dm[2][2] - Dm[0][2] * Dm[2][0];
        C[1][2] = Dm[0][1] * Dm[2][0] - Dm[0][0] * Dm[2][1];
        C[2][0] = Dm[0][1] * Dm[1][2] - Dm[0][2] * Dm[1][1];
        C[2][1] = Dm[0][2] * Dm[1][0] - Dm[0][0] * Dm[1][2];
        C[2][2] = Dm[0][0] * Dm[1][1] - Dm[0][1] * Dm[1][0];
        double I2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b) {
            const double f = (Ds[a][0] * C[b][0] + Ds[a][1] * C[b][1] + Ds[a][2] * C[b][2]) / dm;
            I2 += f * f;
          }
        const double J = ds / dm;
        const double lnJ = log(J);
        const double m = mu[e], l = lam[e];
        en = (dm / 6.0) * (0.5 * m * (I2 - 3.0) - m * lnJ + 0.5 * l * lnJ * lnJ);
      } else {
        bad = 1;
      }
    } else {
      bad = 1;
    }
  }
  // block reduction
  __shared__ double sh_e[kNoallocThreads / 32];
  __shared__ int sh_b[kNoallocThreads / 32];
  __shared__ bool last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    en += __shfl_xor_sync(0xffffffffu, en, o);
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) { sh_e[warp] = en; sh_b[warp] = bad; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double be = 0.0;
    int bb = 0;
    for (int w = 0; w < kNoallocThreads / 32; ++w) { be += sh_e[w]; bb += sh_b[w]; }
    s->partial[blockIdx.x] = be;
    s->invalid[blockIdx.x] = bb;
    __threadfence();
    const unsigned prev = atomicAdd(&s->counter, 1u);
    last = (prev == gridDim.x - 1);
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  double tot = 0.0;
  int tb = 0;
  for (int b = 0; b < (int)gridDim.x; ++b) {  // block order: deterministic
    tot += __ldcg(&s->partial[b]);
    tb += __ldcg(&s->invalid[b]);
  }
  *energy_out = tot;
  *invalid_out = tb;
  s->counter = 0;
}

}  // namespace

extern "C" mls_status mls_elastic_energy_noalloc(int32_t n_verts, int32_t n_tets, const double* rest_xyz,
                                                 const int32_t* tets, const double* mu, const double* lam,
                                                 const double* x, double* energy_out, int32_t* invalid_out,
                                                 void* stream) {
  if (n_verts < 1 || n_tets < 1 || !rest_xyz || !tets || !mu || !lam || !x || !energy_out || !invalid_out)
    return MLS_EINVAL;
  if ((int64_t)n_tets > (int64_t)kNoallocMaxBlocks * kNoallocThreads) return MLS_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return MLS_ECUDA; }
  if (dev < 0 || dev >= kNoallocMaxDevices) return MLS_EINVAL;
  NoallocScratch* s = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return MLS_ECUDA;
      }
      g_scratch_ptr[dev] = (NoallocScratch*)p;
    }
    s = g_scratch_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemsetAsync(&s->counter, 0, sizeof(unsigned int), st) != cudaSuccess) {
    cudaGetLastError();
    return MLS_ECUDA;
  }
  const int nb = (n_tets + kNoallocThreads - 1) / kNoallocThreads;
  k_elastic_energy_noalloc<<<nb, kNoallocThreads, 0, st>>>(n_verts, n_tets, rest_xyz, tets, mu, lam, x, s,
                                                          energy_out, invalid_out);
  if (cudaGetLastError() != cudaSuccess) return MLS_ECUDA;
  return MLS_OK;
}
