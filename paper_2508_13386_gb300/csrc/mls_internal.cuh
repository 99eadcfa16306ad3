// Internal declarations of the sm_103a multilevel timestep library.
//
// Data layout in device memory (n vertices, t tets):
//   vertex vectors      Vec4<T>[n]   (x, y, z, pad) -- one 16 B (float) or
//                                    32 B (double) aligned load per vertex
//   tets                int32 [4][t] SoA, Dm^{-1} double [9][t] SoA,
//                       vol/mu/lam double [t]
//   element gradients   double [12][t] SoA
//   element Hessians    ET [78][t] SoA: the 10 upper 3x3 blocks of the 12x12
//                       (diagonal blocks keep their 6 upper entries)
//   H (3x3 BSR)         sliced ELL with 32 rows per slice ("SELL-32"):
//                       group g holds one block slot of 32 consecutive rows;
//                       col[g*32 + lane], val[g*288 + k*32 + lane] (k = 0..8,
//                       row-major 3x3).  Slot 0 of every row is its diagonal
//                       block; slots past a row's length are padding.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <cstdint>
#include <string>
#include <vector>

#include "mls.h"

namespace mls {

template <typename T> struct alignas(4 * sizeof(T)) Vec4 { T x, y, z, w; };
using Vec4d = Vec4<double>;
using Vec4f = Vec4<float>;

constexpr int kBlock = 256;
constexpr int kSlice = 32;
constexpr int kMaxPartials = 8192;
constexpr int kGalerkinChunk = 128;
// Diagonal-shift retries of a coarse factorisation.  The coarse operator
// only preconditions, so A_c + sigma diag(A_c) serves as well as A_c once
// sigma exceeds the relative indefiniteness that rounding left in it; the
// Newton direction PCG converges to does not depend on the shift.  sigma
// starts at float32 rounding and grows 100x per try.
// Tensor-core trailing updates of the coarse Cholesky (multilevel.cu):
// panel width, bf16 slices per float64 value and bits per slice
constexpr int kOzSlices = 8, kOzBits = 7, kOzPanel = 128;
constexpr int kShiftTries = 4;
constexpr double kShiftFirst = 1e-7;
constexpr double kShiftGrowth = 100.0;
constexpr int kRestrictChunk = 256;
constexpr int kMaxPersistBlocks = 4096;

// offsets of the 10 upper 3x3 blocks inside the 78-value element Hessian
// (order (0,0),(0,1),(0,2),(0,3),(1,1),(1,2),(1,3),(2,2),(2,3),(3,3))
__host__ __device__ constexpr int hess_offset(int a, int b) {
  return a == 0 ? (b == 0 ? 0 : b == 1 ? 6 : b == 2 ? 15 : 24)
       : a == 1 ? (b == 1 ? 33 : b == 2 ? 39 : 48)
       : a == 2 ? (b == 2 ? 57 : 63)
       : 72;
}

template <typename T> __device__ __forceinline__ float to_f(T v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T> __device__ __forceinline__ T from_d(double v);
template <> __device__ __forceinline__ double from_d<double>(double v) { return v; }
template <> __device__ __forceinline__ float from_d<float>(double v) { return (float)v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_d<__nv_bfloat16>(double v) { return __float2bfloat16((float)v); }

template <typename A, typename T> __device__ __forceinline__ A load_as(T v) { return (A)v; }
template <> __device__ __forceinline__ float load_as<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <> __device__ __forceinline__ double load_as<double, __nv_bfloat16>(__nv_bfloat16 v) { return (double)__bfloat162float(v); }

// ---- programmatic dependent launch (chained kernels) ------------------------------------
// A kernel launched with launch_chained() may be scheduled while its
// predecessor in the stream is still running (its launch latency and block
// scheduling overlap the predecessor's tail).  It must call chain_wait()
// before reading or writing anything its predecessor touches; chain_wait()
// returns once the predecessor grid has completed and its writes are
// visible.  chain_release() lets the successor be scheduled.  Both are
// no-ops in a kernel launched the ordinary way.
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_chained(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream,
                                 Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---- deterministic grid-wide sums: block partials, reduced by the last block
struct GridReduce {
  double* partials;        // [K][kMaxPartials]
  unsigned int* counter;   // one counter per reduction slot, left at zero
};

template <int K>
__device__ __forceinline__ void block_sum(double (&v)[K], double (&sh)[K][32]) {
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    v[k] = s;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) sh[k][warp] = v[k];
  }
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = lane < nw ? sh[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      v[k] = s;
    }
  }
  __syncthreads();
}

// sum of base[stride k] over k in [k0, k1), added in index order (so the
// result is the sequential sum's), with eight loads in flight through L2
__device__ __forceinline__ double ordered_sum_ldcg(const double* base, int64_t stride, int k0, int k1) {
  double t = 0.0;
  for (int k = k0; k < k1; k += 8) {
    double v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) v[u] = k + u < k1 ? __ldcg(base + stride * (k + u)) : 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) t += v[u];
  }
  return t;
}

// Sums v over the whole grid.  Returns true in exactly one block (the last
// to arrive), where thread 0 holds the totals in v.  Partials are summed in
// block order, so the result does not depend on scheduling.
template <int K>
__device__ bool grid_sum(double (&v)[K], const GridReduce& gr, int slot) {
  __shared__ double sh[K][32];
  __shared__ bool last;
  block_sum<K>(v, sh);
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) gr.partials[k * kMaxPartials + blockIdx.x] = v[k];
    __threadfence();
    unsigned prev = atomicAdd(gr.counter + slot, 1u);
    last = (prev == (unsigned)nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  // the partials of other blocks are read through L2 (__ldcg), eight loads in
  // flight per thread before they are summed (in block order per thread)
  double acc[K];
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = 0.0;
    const double* base = gr.partials + k * kMaxPartials;
    for (int b0 = threadIdx.x; b0 < nb; b0 += 8 * blockDim.x) {
      double t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int b = b0 + u * blockDim.x;
        t[u] = b < nb ? __ldcg(base + b) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) s += t[u];
    }
    acc[k] = s;
  }
  block_sum<K>(acc, sh);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) v[k] = acc[k];
    gr.counter[slot] = 0;
  }
  return true;
}

// atomic max / min for non-negative doubles through their bit patterns
__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}
__device__ __forceinline__ void atomic_min_nonneg(double* addr, double v) {
  atomicMin((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// PCG scalars kept on the device so iterations run without host round trips.
// rzv/rrv hold r.z and r.r of iteration i in entry i & 1: the kernel that
// opens iteration i writes entry i & 1 while the others read entry
// (i - 1) & 1, the scale of the sums that iteration i produces.
struct PcgScalars {
  double rz, pq, rr, bb, alpha, beta, tol2;
  int iter, max_iter, done;
  double rzv[2], rrv[2];
};

// ---- order-independent sums for the PCG loop -------------------------------------------
// A block's partial x joins a sum as the 128-bit integer round(x 2^(80-e)),
// split into four 32-bit limbs that are added into four 64-bit accumulators
// by fire-and-forget atomics.  Integer addition is associative, so the total
// does not depend on the order in which blocks arrive, and no block waits:
// there is no arrival counter, fence or final pass.  The consumer (a later
// kernel) rebuilds the total from the limbs.  The exponent e comes from an
// estimate of the sum's magnitude that producers and consumer read from the
// same place (the value of the same quantity one iteration earlier), with
// 2^e <= estimate < 2^(e+1): a block partial below 2^(e+30) fits (from there
// up, or not finite, it sets the slot's overflow word), and totals down to
// 2^(e-27) keep all 53 bits.  Each limb accumulates fewer than 2^16 terms below 2^33,
// so no accumulator overflows.  The conversions work on the bit patterns
// with integer instructions: one thread per block runs them, and float64
// instructions issue slowly on this GPU.
constexpr int kFixStride = 4;                  // words between limbs (32 bytes)
constexpr int kFixSlotWords = 5 * kFixStride;  // four limbs + the overflow word
enum { FX_PQ = 0, FX_RR, FX_RZ, FX_KINDS };
constexpr int kFixWords = FX_KINDS * 2 * kFixSlotWords;  // two slots (parities) per kind

__device__ __forceinline__ unsigned long long* fix_slot(unsigned long long* base, int kind, int parity) {
  return base + (kind * 2 + parity) * kFixSlotWords;
}

// floor(log2 x) of a positive normal double below 2^997 (the scale of a
// sum); 0 for anything else
__device__ __forceinline__ int fix_exponent(double estimate) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(estimate);
  const int E = (int)((b >> 52) & 0x7ff);
  return ((b >> 63) || E == 0 || E >= 2020) ? 0 : E - 1023;
}

__device__ __forceinline__ void fix_add(unsigned long long* slot, double x, int e) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0x7ff) {  // infinite or NaN
    atomicOr(slot + 4 * kFixStride, 1ull);
    return;
  }
  if (E == 0) return;  // zero or subnormal: below 2^-1022, under the last place of any scale used
  const unsigned long long m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = E - 1075 + 80 - e;  // |x| 2^(80-e) = m 2^sh
  unsigned __int128 y;
  if (sh >= 0) {
    if (sh > 57) {  // at or beyond 2^110
      atomicOr(slot + 4 * kFixStride, 1ull);
      return;
    }
    y = (unsigned __int128)m << sh;
  } else {
    const int k = -sh;
    if (k > 54) return;  // below half of the last place
    const unsigned long long q = m >> k, rem = m & ((1ull << k) - 1), half = 1ull << (k - 1);
    y = q + ((rem > half || (rem == half && (q & 1ull))) ? 1ull : 0ull);  // nearest, ties to even
  }
  const bool neg = (b >> 63) != 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const unsigned long long l = (unsigned long long)(y >> (32 * k)) & 0xffffffffull;
    if (l) atomicAdd(slot + k * kFixStride, neg ? 0ull - l : l);
  }
}

// raw words of a slot, read through L2 (a later kernel than the producers)
struct FixRaw {
  unsigned long long w[5];
};
__device__ __forceinline__ FixRaw fix_load(const unsigned long long* slot) {
  FixRaw r;
#pragma unroll
  for (int k = 0; k < 5; ++k) r.w[k] = __ldcg(slot + k * kFixStride);
  return r;
}

// the total held by a slot's words, rounded to the nearest double (ties to
// even; outside the normal range 0 or infinity); bad is set if a producer
// overflowed
__device__ __forceinline__ double fix_value(const FixRaw& r, int e, bool& bad) {
  bad = r.w[4] != 0ull;
  unsigned __int128 u = 0;  // limbs are signed: sign-extend, add modulo 2^128
#pragma unroll
  for (int k = 0; k < 4; ++k) u += (unsigned __int128)(__int128)(long long)r.w[k] << (32 * k);
  const bool neg = (__int128)u < 0;
  const unsigned __int128 M = neg ? (unsigned __int128)0 - u : u;
  if (M == 0) return 0.0;
  const unsigned long long hi = (unsigned long long)(M >> 64), lo = (unsigned long long)M;
  const int p = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);  // leading bit
  unsigned long long mant;
  if (p > 52) {
    const int k = p - 52;
    mant = (unsigned long long)(M >> k);
    const unsigned __int128 rem = M & ((((unsigned __int128)1) << k) - 1), half = ((unsigned __int128)1) << (k - 1);
    if (rem > half || (rem == half && (mant & 1ull))) ++mant;
  } else {
    mant = (unsigned long long)M << (52 - p);
  }
  int field = p + e - 80 + 1023;
  if (mant >> 53) {
    mant >>= 1;
    ++field;
  }
  const unsigned long long sign = neg ? (1ull << 63) : 0ull;
  if (field <= 0) return __longlong_as_double((long long)sign);
  if (field >= 2047) return __longlong_as_double((long long)(sign | (0x7ffull << 52)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)field << 52) | (mant & ((1ull << 52) - 1))));
}

__device__ __forceinline__ void fix_clear(unsigned long long* slot) {
#pragma unroll
  for (int k = 0; k < 5; ++k) slot[k * kFixStride] = 0ull;
}

// double -> float, nearest with ties to even, by integer instructions
// (outside the normal float range: 0 or infinity)
__device__ __forceinline__ float dbl_to_flt(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 63) << 31;
  const int E = (int)((b >> 52) & 0x7ff) - 1023;
  if (E < -126) return __uint_as_float(sign);
  if (E > 127) return __uint_as_float(sign | 0x7f800000u);
  const unsigned long long m = b & ((1ull << 52) - 1), rem = m & ((1ull << 29) - 1), half = 1ull << 28;
  unsigned mant = (unsigned)(m >> 29);
  unsigned fe = (unsigned)(E + 127);
  if (rem > half || (rem == half && (mant & 1u))) ++mant;
  if (mant >> 23) {
    mant = 0;
    ++fe;
  }
  if (fe >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | (fe << 23) | mant);
}

// tests on the bit patterns of doubles (no float64 instructions)
__device__ __forceinline__ bool dbl_finite(double x) {
  return (((unsigned long long)__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool dbl_positive(double x) {  // > 0 and finite
  const long long b = __double_as_longlong(x);
  return b > 0 && dbl_finite(x);
}
// a <= b for non-negative finite doubles: their bit patterns order like the values
__device__ __forceinline__ bool dbl_le_nonneg(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }

// x 2^d for a normal double x by moving its exponent field (0 or infinity
// when the result leaves the normal range), integer instructions only
__device__ __forceinline__ double dbl_scale2(double x, int d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  if (E == 0 || E == 0x7ff) return x;
  const int F = E + d;
  const unsigned long long sign = b & (1ull << 63);
  if (F <= 0) return __longlong_as_double((long long)sign);
  if (F >= 0x7ff) return __longlong_as_double((long long)(sign | (0x7ffull << 52)));
  return __longlong_as_double((long long)((b & ~(0x7ffull << 52)) | ((unsigned long long)F << 52)));
}

// a / b in the solve precision: for float vectors a float division after
// both operands are scaled by the same power of two (b to [1, 2)), so dot
// products beyond the float range still give their ratio (float64 division
// issues slowly); float64 division for float64 vectors
template <typename VT>
__device__ __forceinline__ VT ratio(double a, double b) {
  if constexpr (sizeof(VT) == 4) {
    const int eb = (int)(((unsigned long long)__double_as_longlong(b) >> 52) & 0x7ff);
    return dbl_to_flt(dbl_scale2(a, 1023 - eb)) / dbl_to_flt(dbl_scale2(b, 1023 - eb));
  } else {
    return a / b;
  }
}

// The state that opens PCG iteration i: r.z and r.r of the iterate, the
// step beta_i = rz_i / rz_{i-1} (0 for i = 0) in the solve precision, and
// the stopping decision (1 converged, 2 iteration cap, 3 breakdown or
// non-finite value).
template <typename VT>
struct PcgHead {
  double rz, rr;
  VT beta;
  int done;
};
struct PcgHeadRaw {
  FixRaw rz, rr;
};
__device__ __forceinline__ PcgHeadRaw pcg_head_load(const unsigned long long* fix, int i) {
  PcgHeadRaw raw;
  raw.rz = fix_load(fix_slot(const_cast<unsigned long long*>(fix), FX_RZ, i & 1));
  raw.rr = fix_load(fix_slot(const_cast<unsigned long long*>(fix), FX_RR, i & 1));
  return raw;
}
template <typename VT>
__device__ __forceinline__ PcgHead<VT> pcg_head(const PcgScalars* S, const PcgHeadRaw& raw, int i) {
  PcgHead<VT> h;
  bool bad = false;
  if (i == 0) {
    h.rz = S->rzv[0];
    h.rr = S->rrv[0];
    h.beta = VT(0);
  } else {
    const double rzp = S->rzv[(i - 1) & 1], rrp = S->rrv[(i - 1) & 1];
    bool b1, b2;
    h.rz = fix_value(raw.rz, fix_exponent(rzp), b1);
    h.rr = fix_value(raw.rr, fix_exponent(rrp), b2);
    h.beta = ratio<VT>(h.rz, rzp);
    bad = b1 || b2;
  }
  h.done = 0;
  if (bad || !dbl_finite(h.rr)) h.done = 3;
  else if (dbl_le_nonneg(h.rr, S->tol2)) h.done = 1;
  else if (!dbl_positive(h.rz)) h.done = 3;
  else if (i >= S->max_iter) h.done = 2;
  return h;
}
// The same loads spread over the lanes of one warp, so that they take one
// round trip instead of a chain: lanes 0-4 and 5-9 read the r.z and r.r
// slots, lanes 10-16 the stop flag and the scalars the decision needs, and
// every lane gets every value by shuffles.  Call with a whole warp.
struct PcgOpen {
  FixRaw rz, rr;
  double rzp, rrp, tol2, rz0, rr0;
  int max_iter, done;
};
__device__ __forceinline__ PcgOpen pcg_open_load_warp(const unsigned long long* fix, const PcgScalars* S, int i) {
  const int lane = threadIdx.x & 31;
  const unsigned long long* rzs = fix_slot(const_cast<unsigned long long*>(fix), FX_RZ, i & 1);
  const unsigned long long* rrs = fix_slot(const_cast<unsigned long long*>(fix), FX_RR, i & 1);
  const int ip = (i - 1) & 1;
  unsigned long long w = 0ull;
  if (lane < 5) w = __ldcg(rzs + lane * kFixStride);
  else if (lane < 10) w = __ldcg(rrs + (lane - 5) * kFixStride);
  else if (lane == 10) w = (unsigned long long)(unsigned)__ldcg(&S->done);
  else if (lane == 11) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rzv[ip]));
  else if (lane == 12) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rrv[ip]));
  else if (lane == 13) w = (unsigned long long)__double_as_longlong(__ldcg(&S->tol2));
  else if (lane == 14) w = (unsigned long long)(unsigned)__ldcg(&S->max_iter);
  else if (lane == 15) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rzv[0]));
  else if (lane == 16) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rrv[0]));
  PcgOpen o;
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    o.rz.w[k] = __shfl_sync(0xffffffffu, w, k);
    o.rr.w[k] = __shfl_sync(0xffffffffu, w, 5 + k);
  }
  o.done = (int)__shfl_sync(0xffffffffu, w, 10);
  o.rzp = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 11));
  o.rrp = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 12));
  o.tol2 = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 13));
  o.max_iter = (int)__shfl_sync(0xffffffffu, w, 14);
  o.rz0 = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 15));
  o.rr0 = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 16));
  return o;
}
// pcg_head() from the values pcg_open_load_warp() read
template <typename VT>
__device__ __forceinline__ PcgHead<VT> pcg_head_open(const PcgOpen& o, int i) {
  PcgHead<VT> h;
  bool bad = false;
  if (i == 0) {
    h.rz = o.rz0;
    h.rr = o.rr0;
    h.beta = VT(0);
  } else {
    bool b1, b2;
    h.rz = fix_value(o.rz, fix_exponent(o.rzp), b1);
    h.rr = fix_value(o.rr, fix_exponent(o.rrp), b2);
    h.beta = ratio<VT>(h.rz, o.rzp);
    bad = b1 || b2;
  }
  h.done = 0;
  if (bad || !dbl_finite(h.rr)) h.done = 3;
  else if (dbl_le_nonneg(h.rr, o.tol2)) h.done = 1;
  else if (!dbl_positive(h.rz)) h.done = 3;
  else if (i >= o.max_iter) h.done = 2;
  return h;
}

// written once per iteration (block 0 of the opening kernel): the state for
// later kernels and the host, and the PQ slot of iteration i - 1 cleared
template <typename VT>
__device__ __forceinline__ void pcg_head_publish(PcgScalars* S, unsigned long long* fix, int i, const PcgHead<VT>& h) {
  if (i > 0) {
    S->rzv[i & 1] = h.rz;
    S->rrv[i & 1] = h.rr;
    fix_clear(fix_slot(fix, FX_PQ, (i - 1) & 1));
  }
  S->rz = h.rz;
  S->rr = h.rr;
  S->iter = i;
  if (h.done) S->done = h.done;
}

// Reduction slots (one counter each)
enum { RS_PCG_PQ = 0, RS_PCG_RR, RS_PCG_RZ, RS_ENERGY, RS_MISC, RS_GRAD, RS_CONTACT, RS_COUNT };

struct Basis {
  int m = 0;                  // handles
  int nnz = 0;                // vertex-handle pairs
  int* vrow = nullptr;        // [n+1]  per-vertex CSR
  int* vh = nullptr;          // [nnz]  handle
  double* vphi = nullptr;     // [nnz]
  int* hrow = nullptr;        // [m+1]  per-handle CSR (transpose)
  int* hv = nullptr;          // [nnz]  vertex
  double* hphi = nullptr;     // [nnz]
  double* origins = nullptr;  // [m][3]
  // Galerkin structure
  int* yrow = nullptr;        // [n+1] CSR of handles reachable from row v through H
  int* yh = nullptr;          // [ny] handle of each (v, j) pair
  int64_t ny = 0;
  int16_t* yslot = nullptr;   // [n_slots * maxk] local index into row v's Y list per (slot, basis entry)
  int maxk = 0;               // max handles per vertex
  int maxkv = 0;              // max K_v: handles reachable from one row of H
  int* hn_row = nullptr;      // [m+1] coarse block-row neighbours (CSR)
  int* hn = nullptr;          // [nb] neighbour handle
  int nb = 0;
  int* ent_ptr = nullptr;     // [nb+1] entries of each coarse block (i, hn[s])
  int* ent_y = nullptr;       // [nent] index of Y_vj
  int* ent_v = nullptr;       // [nent] vertex v in supp(i)
  double* ent_phi = nullptr;  // [nent] phi_i(v)
  int64_t nent = 0;
  int* ypair_row = nullptr;   // [ny] row v of each (v, j) pair
  int* chunk_ptr = nullptr;   // [nb+1] first chunk of each coarse block
  int* chunk_beg = nullptr;   // [nchunk] first entry of each chunk
  int* slot_row = nullptr;    // [nb] coarse block row i of each block
  int nchunk = 0;
  void* vcoef = nullptr;      // [nnz] Vec4 (phi, phi a) per (vertex, handle), solve precision
  void* hcoef = nullptr;      // [nnz] same, handle-major
  int* rchunk_handle = nullptr;  // restriction chunks
  int* rchunk_beg = nullptr;
  int* rchunk_ptr = nullptr;  // [m+1]
  double* rpart = nullptr;    // [nrchunk][12]
  unsigned* rcount = nullptr; // [m] arrivals per handle, left at zero
  int nrchunk = 0;
  std::vector<int> h_vrow, h_hrow, h_vh;
  std::vector<double> h_vphi, h_origins;
};

// ---- lagged point-plane friction (Eq. IP, term D) ------------------------------------
// The IPC-style friction of a vertex v against the ground plane (unit normal n,
// offset o), lagged at x^t once per timestep:
//   lam_v = -kappa b'(n . x_v^t - o)   the normal force at x^t (0 outside (0, dhat))
//   u_v   = (I - n n^T)(x_v - x_v^t)   the tangential slip over the step, y = |u_v|
//   D_v   = mu lam_v f0(y)             with the C1 mollifier of width eps = eps_v h:
//   f0(y) = -y^3 / (3 eps^2) + y^2 / eps + eps / 3,   f1 = f0' = 2y/eps - y^2/eps^2   (y < eps)
//   f0(y) = y,                                        f1 = 1                         (y >= eps)
// so grad D_v = mu lam_v (f1(y) / y) u_v and the Hessian block is
//   mu lam_v [ (f1/y) (I - n n^T) + (f1' - f1/y) u^ u^T ],  u^ = u_v / y,
// positive semi-definite (f1' >= 0, f1/y > 0); at y = 0 both factors are 2/eps.
__device__ __forceinline__ double fric_lambda(double d_t, double dhat, double kappa) {
  if (d_t >= dhat || d_t <= 0.0) return 0.0;
  const double r = d_t - dhat;
  return -kappa * (-2.0 * r * log(d_t / dhat) - r * r / d_t);
}
// tangential slip u (returned in u[3]) and its length
__device__ __forceinline__ double fric_slip(const Vec4d& xv, const Vec4d& xtv, double n0, double n1, double n2,
                                            double (&u)[3]) {
  const double dx = xv.x - xtv.x, dy = xv.y - xtv.y, dz = xv.z - xtv.z;
  const double un = n0 * dx + n1 * dy + n2 * dz;
  u[0] = dx - un * n0; u[1] = dy - un * n1; u[2] = dz - un * n2;
  return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}
// f1(y) / y, finite at y = 0
__device__ __forceinline__ double fric_ratio(double y, double eps) {
  return y < eps ? 2.0 / eps - y / (eps * eps) : 1.0 / y;
}
// f1'(y)
__device__ __forceinline__ double fric_slope(double y, double eps) {
  return y < eps ? 2.0 / eps - 2.0 * y / (eps * eps) : 0.0;
}
__device__ __forceinline__ double fric_f0(double y, double eps) {
  return y < eps ? -y * y * y / (3.0 * eps * eps) + y * y / eps + eps / 3.0 : y;
}

}  // namespace mls

struct mls_mlp;

namespace mls {
// Mesh-mesh contact (contact.cu): the surface primitives of the bodies, the
// hashed grid of the broad phase, the candidate pairs and the coupling
// blocks of the last assembly
struct ContactState {
  bool on = false;
  int nf = 0, ne = 0, nsv = 0;       // boundary faces, their edges, surface vertices
  int4* faces = nullptr;             // [nf] {a, b, c, body}
  int4* edges = nullptr;             // [ne] {a, b, body, 0}
  int2* sverts = nullptr;            // [nsv] {v, body}
  int* row_len0 = nullptr;           // [n] row lengths of H's element pattern
  double dhat = 1e-3, kappa = 1e5;   // barrier of the pairs
  double cell0 = 0.0;                // mean rest length of the surface edges
  int spare = 0;                     // spare block slots per surface-vertex row
  int nbody = 0;                     // bodies (largest label + 1)
  unsigned long long* bbox = nullptr;  // per-body boxes of the broad phase: [3 nbody] low, [3 nbody] high keys
  // hashed grid: bucket heads, entries {primitive, ix, iy, iz} and chain links
  int* head = nullptr;
  int hbits = 0;
  int4* ent = nullptr;
  int* next = nullptr;
  int64_t ecap = 0;
  double* boxes = nullptr;           // [nf + ne][6] grown boxes of the entered primitives
  int* cnt = nullptr;                // device counters
  int* cnt_host = nullptr;           // pinned mirror
  int2* pt = nullptr;                // point-triangle pairs {v, face} within dhat at the assembly iterate
  int2* ee = nullptr;                // edge-edge pairs {edge, edge}
  int64_t pcap = 0;
  int npt = 0, nee = 0;
  int2* spt = nullptr;               // candidates over the segment x -> x + d (CCD, line search)
  int2* see = nullptr;
  int64_t scap = 0;
  int nspt = 0, nsee = 0;
  bool sweep_valid = false;
  const void* sweep_x = nullptr;
  const void* sweep_d = nullptr;
  double* pg = nullptr;              // [pbuf_cap][12] barrier gradient of each pair
  double* pH = nullptr;              // [pbuf_cap][144] its projected Hessian
  int pbuf_cap = 0;
  unsigned long long* ckey = nullptr;  // coupling table: key (i << 32 | j), open addressing
  double* cval = nullptr;              // [ccap][9] barrier blocks (kappa, no h^2)
  int ccap = 0;
  int4* xc = nullptr;                // cross-body couplings {i, j, slot of H, 0}
  int xcap = 0;
  int nxc = 0;
  Vec4d* cgrad = nullptr;            // [n] barrier and friction gradient of the pairs (no h^2)
  double* ccd = nullptr;             // device: smallest CCD fraction
  std::vector<int> h_body;
  // friction between bodies, lagged at x^t: the pairs within dhat there
  int2* fpt = nullptr;               // broad-phase output at x^t
  int2* fee = nullptr;
  int64_t fbcap = 0;
  int4* fv = nullptr;                // [fcap] each lagged pair's four vertices
  double* fw = nullptr;              // [fcap][8] w[4], n[3], mu lambda
  int fcap = 0;
  int nfr = 0;                       // lagged pairs of the current step
};
}  // namespace mls

struct mls_ctx {
  mls_options opt{};
  cudaStream_t stream = nullptr;
  std::string err;
  int device = 0;

  // mesh
  int n = 0, t = 0;
  int* tets = nullptr;       // [4][t]
  double* Dminv = nullptr;   // [9][t]
  double* vol = nullptr;     // [t]
  double* mu = nullptr;      // [t]
  double* lam = nullptr;     // [t]
  double* mass = nullptr;    // [n]
  uint8_t* pinned = nullptr; // [n]
  mls::Vec4d* X = nullptr;   // [n] rest positions

  // sparsity of H (SELL-32)
  int n_slices = 0;
  int64_t n_groups = 0;            // slot groups of 32
  int* slice_ptr = nullptr;        // [n_slices + 1] first group of each slice
  int* group_slice = nullptr;      // [n_groups]
  int* col = nullptr;              // [n_groups * 32]
  int* row_len = nullptr;          // [n]
  int* asm_ptr = nullptr;          // [n_groups * 32 + 1]
  int* asm_code = nullptr;         // [16 t] (e * 16 + a * 4 + b)
  int* vt_ptr = nullptr;           // [n + 1]
  int* vt_code = nullptr;          // [4 t] (e * 4 + a)
  int64_t nnzb = 0;                // real (non-padding) blocks
  double mass_min = 0.0;           // smallest lumped vertex mass
  std::vector<int> h_slice_ptr, h_row_len, h_col;
  std::vector<int> h_tets;         // [t][4] host copy (the pattern is rebuilt with contact slots)
  mls::ContactState cs;            // mesh-mesh contact

  // per-timestep / per-iteration state
  double h = 1.0 / 60.0;           // step of the implicit-Euler potential the Newton loop minimises
                                   // (2 h_step / 3 for BDF2: its potential carries (4/9) h_step^2)
  double h_step = 1.0 / 60.0;      // the timestep itself (stopping scale, friction mollifier width)
  mls::Vec4d* xk = nullptr;        // current iterate
  mls::Vec4d* xt = nullptr;        // x^t
  mls::Vec4d* xtil = nullptr;      // predictor
  mls::Vec4d* dir = nullptr;       // Newton direction (float64)
  mls::Vec4d* grad = nullptr;      // gradient (float64)
  mls::Vec4d* tmp4 = nullptr;      // zero vector (float64), restored after scratch use
  double* stage = nullptr;         // [3][n][3] staging for host-pointer timesteps
  double* egrad = nullptr;         // [12][t]
  void* ehess = nullptr;           // [78][t] element precision
  void* ehess_lag = nullptr;       // element Hessians of the last H_lag refresh (hessian_lag)
  void* hval_lag = nullptr;        // H_lag values and its block-Jacobi inverse
  void* dinv_lag = nullptr;
  int lag_age = 0;                 // Newton iterations since the last refresh
  int lag_nalpha = 0;              // line-search step sizes since the refresh (up to 3 kept)
  double lag_alpha[3] = {1.0, 1.0, 1.0};
  void* hval = nullptr;            // [n_groups * 288] storage precision
  void* dinv = nullptr;            // [n][9] solve precision
  void* vb = nullptr;              // PCG vectors in solve precision: b, x, r, z, p, q, w
  void* vx = nullptr;
  void* vr = nullptr;
  void* vz = nullptr;
  void* vp = nullptr;
  void* vq = nullptr;
  void* vw = nullptr;
  void* vz2 = nullptr;             // preconditioned residual of the multiplicative cycle
  double* cub_scale = nullptr;     // device [t]: cubature factor per element on its elastic Hessian (nullable)
  void* hval_cub = nullptr;        // the cubature H the coarse operator is built from (with cub_scale)
  double omega_eff = 0.5;          // damping the two-level cycle applies (opt.omega or the automatic choice)
  double omega_lmax = 0.0;         // the automatic choice's estimate of lambda_max(D^{-1} H)
  double* lz = nullptr;            // device: Lanczos alpha[kLanczosSteps], beta[kLanczosSteps + 1]
  mls::PcgScalars* pcg = nullptr;  // device
  unsigned long long* pcg_fix = nullptr;  // device: [kFixWords] order-independent PCG sums
  double* persist_part = nullptr;  // [kMaxPersistBlocks][4] persistent-PCG block partials
  void* persist_bar = nullptr;     // persistent-PCG grid barrier state
  int persist_blocks = 0;          // cooperative grid size (0 = not yet sized)
  int persist_bps = -1;            // (blocks per SM, precision, cycle) it was sized for
  mls::PcgScalars* pcg_host = nullptr;  // pinned
  double* dscal = nullptr;         // device scalars [16]
  double* dscal_host = nullptr;    // pinned [16]
  mls::GridReduce red{};
  bool assembled = false;

  // forces
  double grav[3] = {0.0, 0.0, -9.81};
  int contact = 0;
  double pn[3] = {0.0, 0.0, 1.0};
  double po = 0.0, dhat = 1e-3, kappa = 1e5;
  double fric_mu = 0.0;            // lagged point-plane friction coefficient (0: no friction term)
  double fric_eps_v = 1e-3;        // friction mollifier width as a velocity (width eps_v h_step)

  // basis / coarse level
  mls::Basis basis;
  bool has_basis = false;
  double* Ac = nullptr;            // [r][r] float64 Galerkin operator, then its Cholesky factor
  void* Linv = nullptr;            // [r][r] W = L^{-1} in solve precision (lower)
  void* LinvT = nullptr;           // [r][r] W^T (upper)
  void* Ainv = nullptr;            // [r][r] W^T W = (U^T H U)^{-1}, dense, solve precision
  double* Acopy = nullptr;         // [r][r] copy of the operator before factorisation
  void* yval = nullptr;            // [ny][36] H U blocks (solve precision)
  void* gpart = nullptr;           // [nchunk][144] Galerkin chunk partial sums
  void* cvec = nullptr;            // [r] coarse vectors (solve precision)
  void* cvec2 = nullptr;
  __nv_bfloat16* oz_fwd = nullptr;  // [r][8 x 128] bf16 slices of a Cholesky panel (tensor-core update)
  int* oz_e = nullptr;              // [r] row exponents of the panel
  int* umma_err = nullptr;          // set by a tensor-core product whose bounded wait gave up
  double* sms_buf = nullptr;        // Alg. 2 subspace PCG: [r] q, res, z, p and the [m][144] block inverses
  void* sms_cg = nullptr;           // its scalars
  double* sms_m = nullptr;          // [r][12] U^T H U T (the affine level's operator before T^T)
  bool galerkin_ready = false;      // Acopy holds U^T H U of the current iterate (direction 2)
  bool coarse_ready = false;
  bool coarse_fallback = false;    // this Newton iteration preconditions with block Jacobi (coarse factor failed)
  int64_t coarse_shift_count = 0;  // diagonal-shift retries of the coarse factorisation so far
  double coarse_sigma = 0.0;       // relative diagonal shift of the current coarse factor (0: none)
  int coarse_age_steps = 0;       // timesteps begun since the coarse factor was built
  int coarse_ref_iters = 0;       // PCG iterations of a step's first solve after that build
  bool coarse_ref_pending = false; // the next step's first solve sets coarse_ref_iters
  bool coarse_stale = false;      // a lagged factor slowed PCG down: rebuild next iteration
  int* chol_info = nullptr;        // device: first non-positive pivot + 1, or 0
  double* chol_tinv = nullptr;     // [tiles][32][32] inverses of the diagonal factor tiles

  // learned warm start (coarse projection with U^T M U, history, features)
  double* Am = nullptr;            // [r][r] U^T M U, factored in place
  void* Wm = nullptr;              // inverse factor of U^T M U (solve precision)
  void* WmT = nullptr;
  void* ws_c = nullptr;            // [r] solve-precision scratch
  void* ws_c2 = nullptr;
  void* ws_tmp = nullptr;
  double* ws_hist = nullptr;       // [3][r] q^t, q^{t-1}, q^{t-2}
  double* ws_qg = nullptr;         // [r] coarse coordinates of h^2 g
  double* ws_qtilde = nullptr;     // [r] q(x_tilde)
  double* ws_qnext = nullptr;      // [r] scratch projection
  float* ws_feat = nullptr;        // [3r] features of the current step
  float* ws_target = nullptr;      // [r] realised coarse increment of the last step
  float* ws_pred = nullptr;        // [r] predicted increment
  mls_mlp* ws_mlp = nullptr;       // attached network (not owned)
  bool ws_ready = false, ws_enabled = false, ws_hist_valid = false;
  bool ws_record = false;          // record training targets (keeps H(x_tilde))
  void* ws_hsave = nullptr;        // copy of H's values at the first Newton iterate
  std::vector<double> h_mass, h_X; // host copies for assembling U^T M U
  std::vector<uint8_t> h_pinned;   // host copy of the Dirichlet mask

  // kernel-class timing
  uint32_t prof_mask = 0;
  std::vector<cudaEvent_t> prof_pool;
  std::vector<std::pair<int, int>> prof_pending;  // (class, first event of the pair)
  double prof_ms[MLS_PROF_COUNT] = {};
  int64_t prof_n[MLS_PROF_COUNT] = {};

  int64_t launches = 0;            // kernels launched by this context
  std::vector<void*> allocs;       // every device allocation, freed by mls_destroy
  std::vector<void*> host_allocs;  // pinned host allocations
};

namespace mls {

// kernel-class timing: prof_begin returns a token (or -1 when the class is off)
int prof_begin(mls_ctx* ctx, int cls);
void prof_end(mls_ctx* ctx, int token);
void prof_flush(mls_ctx* ctx);  // call after the stream is synchronised

// allocation helpers (host side; record for cleanup)
mls_status dalloc(mls_ctx* ctx, void** p, size_t bytes);
void dfree(mls_ctx* ctx, void* p);
mls_status fail(mls_ctx* ctx, mls_status st, const std::string& msg);
mls_status cuda_check(mls_ctx* ctx, cudaError_t e, const char* what);

int solve_bytes(const mls_ctx* ctx);     // bytes per scalar of PCG vectors
int storage_bytes(const mls_ctx* ctx);   // bytes per scalar of H values
int element_bytes(const mls_ctx* ctx);   // bytes per scalar of element Hessians

// kernels launched from the host code (each file exposes launchers)
mls_status launch_eval_elements(mls_ctx* ctx, const Vec4d* x, double* energy_out);
mls_status launch_expand_hessian(mls_ctx* ctx, double* hess_out);
mls_status launch_gather_grad(mls_ctx* ctx, const Vec4d* x, double* gnorm2_out);
mls_status launch_assemble(mls_ctx* ctx, const Vec4d* x);
mls_status launch_energy(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, double* E,
                         int* infeasible);
mls_status launch_ccd(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double* alpha);
mls_status launch_norms(mls_ctx* ctx, const Vec4d* d, double* dinf, double* xdisp_inf);
mls_status launch_axpy_state(mls_ctx* ctx, Vec4d* x, const Vec4d* d, double alpha);
mls_status launch_diff_state(mls_ctx* ctx, const Vec4d* a, const Vec4d* b, Vec4d* out);   // out = a - b
mls_status launch_xpay_state(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, Vec4d* out);  // x + alpha d
mls_status launch_predictor(mls_ctx* ctx, const double* x, const double* v, double dt);
// BDF2 predictor from (x^t, v^t) and (x^{t-1}, v^{t-1}) with timestep dt
mls_status launch_predictor_bdf2(mls_ctx* ctx, const double* x, const double* v, const double* x_prev,
                                 const double* v_prev, double dt);
mls_status launch_pack(mls_ctx* ctx, const double* src, Vec4d* dst);
mls_status launch_unpack(mls_ctx* ctx, const Vec4d* src, double* dst);
mls_status launch_disp_out(mls_ctx* ctx, double* dx_out);

mls_status launch_spmv(mls_ctx* ctx, const void* x, void* y);  // solve-precision vectors
mls_status launch_assemble_cubature(mls_ctx* ctx, const Vec4d* x);  // cubature H into hval_cub
constexpr int kLanczosSteps = 20;  // Lanczos steps of the automatic smoother damping
// largest eigenvalue of the symmetric tridiagonal matrix with diagonal d[0..k-1]
// and off-diagonal e[0..k-2] (Sturm-count bisection), from above to rounding
double tridiag_max_eig(const double* d, const double* e, int k);
mls_status launch_spmv_values(mls_ctx* ctx, const void* values, const void* x, void* y);
mls_status launch_to_solve(mls_ctx* ctx, const Vec4d* src, void* dst, double scale);
mls_status launch_from_solve(mls_ctx* ctx, const void* src, Vec4d* dst);
mls_status launch_add_solve(mls_ctx* ctx, void* y, const void* x);       // y += x, solve precision      // zero on Dirichlet vertices
mls_status launch_from_solve_raw(mls_ctx* ctx, const void* src, Vec4d* dst);  // no masking
mls_status pcg_solve(mls_ctx* ctx, double rtol, int max_iter, int* iters, double* rel_res);
mls_status launch_residual(mls_ctx* ctx, const void* b, const void* x, void* out, const PcgScalars* S);
mls_status launch_persistent_pcg(mls_ctx* ctx, int cycle, int iters);
mls_status precond_apply(mls_ctx* ctx, const void* r, void* z);

mls_status basis_upload(mls_ctx* ctx, int m, const double* origins, const int* vrow,
                        const int* handle, const double* phi);
mls_status launch_prolong(mls_ctx* ctx, const void* q, void* w, bool accumulate);
mls_status launch_restrict(mls_ctx* ctx, const void* r, void* q);
mls_status build_coarse(mls_ctx* ctx);

// C = epilogue(A B^T) on the tensor cores (umma.cu): A [M][lda], B [N][ldb]
// bf16 row-major (pitches multiples of 8 elements, 16-byte aligned), C
// float32 [M][ldc]; *err (device) is set if a bounded wait gave up
struct GemmEpilogue {
  const float* bias = nullptr;    // [N]: + bias[n]
  int relu = 0;                   // then max(., 0)
  const float* mask = nullptr;    // [M][ldc]: then zero where mask <= 0
  const float* oscale = nullptr;  // [N]: then x oscale[n] + oshift[n]
  const float* oshift = nullptr;
  __nv_bfloat16* out16 = nullptr;   // [M][ld16]: the result rounded to bf16 as well
  int ld16 = 0;
  __nv_bfloat16* out16t = nullptr;  // [N][ld16t]: its transpose rounded to bf16
  int ld16t = 0;
  // float64 accumulation instead of the float32 store (the slice products of
  // the emulated float64 product): acc64[m][n] += sign x 2^(ea[m] + eb[n] -
  // ebias) x result, exact scaling and one float64 addition
  double* acc64 = nullptr;
  int ld64 = 0;
  const int* ea = nullptr;
  const int* eb = nullptr;
  int ebias = 0;
  double sign = 1.0;
  int lower = 0;                    // only tiles that meet the lower triangle n <= m
};
mls_status gemm_bf16_tn(cudaStream_t stream, int M, int N, int K, const __nv_bfloat16* A, int lda,
                        const __nv_bfloat16* B, int ldb, float* C, int ldc, const GemmEpilogue& ep, int* err);
// A[i][j] -= (L21 L21^T)[i][j], j <= i < n, on the tensor cores from the
// bf16 slices of L21's rows (umma.cu; slicing in multilevel.cu)
mls_status ozaki_syrk(cudaStream_t stream, int n, const __nv_bfloat16* fwd, int opitch, const int* e, double* A,
                      int lda, int* err);
mls_status build_galerkin(mls_ctx* ctx);   // U^T H U into the dense Ac only (no factorisation)
mls_status coarse_apply(mls_ctx* ctx, const void* c_in, void* c_out);
mls_status sms_pcg(mls_ctx* ctx, const void* b, double rtol, int max_iter, int* iters);
mls_status build_coarse_unfactored(mls_ctx* ctx);
mls_status launch_assemble_lagged(mls_ctx* ctx, const Vec4d* x);
mls_status affine_operator(mls_ctx* ctx, const double om[3]);
// mesh-mesh contact (contact.cu)
mls_status build_pattern(mls_ctx* ctx, const std::vector<int>* spare);
mls_status contact_assemble(mls_ctx* ctx, const Vec4d* x);           // pairs, gradient, coupling blocks at x
mls_status contact_merge(mls_ctx* ctx, void* val, void* dinv, bool record);  // coupling blocks into H
mls_status contact_energy(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, double* E, int* infeasible);
mls_status contact_ccd(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double* t);
mls_status contact_galerkin(mls_ctx* ctx, const void* val);          // cross-body U_i^T H_ij U_j into Ac
void contact_invalidate(mls_ctx* ctx);                               // x or d changed: sweep again
mls_status contact_friction_lag(mls_ctx* ctx);                       // friction pairs and frames at x^t
void contact_free(mls_ctx* ctx);
mls_status warm_start_begin(mls_ctx* ctx, int* used);
mls_status warm_start_first_iteration(mls_ctx* ctx);
mls_status warm_start_end(mls_ctx* ctx);

}  // namespace mls
