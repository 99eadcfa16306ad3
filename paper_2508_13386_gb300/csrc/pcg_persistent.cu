// Persistent PCG: the whole preconditioned CG iteration loop (Eq. 5 solve
// with block Jacobi or the two-level cycle of Sec. 3.7) in one cooperative
// launch per chunk of iterations.  The phases of an iteration (product,
// vector update, residual, restriction, the two coarse triangular products,
// prolongation, post-smoothing) are separated by a grid-wide barrier instead
// of kernel boundaries: at this size (73K vertex rows) every phase is
// latency-bound, and per-kernel launch, ramp-up and reduction tails dominated
// the separate-kernel loop.
//
// Reductions: each block writes a partial sum, and after the barrier every
// block adds all partials in block order, so all blocks hold the identical
// scalar (alpha, beta, |r|^2) without a second launch or atomics.
//
// The barrier is sense-reversing with a bounded spin: a block that waits more
// than kBarrierSpinLimit polls sets an error flag and every block leaves the
// kernel; the host reports MLS_ETIMEOUT.  The launch is cooperative, so all
// blocks are co-resident and the limit is never reached in normal operation.
#include "mls_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace mls {

constexpr int kPersistThreads = 256;
static_assert(kPersistThreads == kRestrictChunk, "one restriction chunk per block pass");
constexpr unsigned kBarrierSpinLimit = 1u << 26;

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
  int error;
};

__device__ __forceinline__ bool grid_barrier(GridBarrier* bar, unsigned nblocks,
                                             unsigned spin_limit = kBarrierSpinLimit) {
  __syncthreads();
  __shared__ int s_err;
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = &bar->gen;
    const unsigned g = *vgen;
    __threadfence();
    if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
      bar->count = 0;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      unsigned spins = 0;
      while (*vgen == g) {
        if (++spins > spin_limit || *(volatile int*)&bar->error) {
          atomicExch(&bar->error, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    s_err = *(volatile int*)&bar->error;
  }
  __syncthreads();
  return s_err == 0;
}

// Loads of vectors that other blocks write inside this kernel go through L2
// (__ldcg): L1 is not coherent across SMs.
__device__ __forceinline__ Vec4f ldv(const Vec4f* p) {
  const float4 v = __ldcg(reinterpret_cast<const float4*>(p));
  return Vec4f{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ Vec4d ldv(const Vec4d* p) {
  const double2 a = __ldcg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldcg(reinterpret_cast<const double2*>(p) + 1);
  return Vec4d{a.x, a.y, b.x, b.y};
}

// block-wide sum of K doubles; thread 0 gets the totals
template <int K>
__device__ __forceinline__ void block_sum_p(double (&v)[K]) {
  __shared__ double sh[K][kPersistThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) {
      double s = 0.0;
      for (int w = 0; w < kPersistThreads / 32; ++w) s += sh[k][w];
      v[k] = s;
    }
  }
  __syncthreads();
}

template <typename VT>
struct PersistArgs {
  int n, n_slices;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ col;
  const int* __restrict__ row_len;
  const VT* __restrict__ dinv;
  VT omega;
  Vec4<VT>* x;
  Vec4<VT>* r;
  Vec4<VT>* p;
  Vec4<VT>* q;
  Vec4<VT>* z1;
  Vec4<VT>* zf;
  Vec4<VT>* t;
  // basis
  int m;
  const int* __restrict__ vrow;
  const int* __restrict__ vh;
  const void* __restrict__ vcoef;
  const int* __restrict__ hrow;
  const int* __restrict__ hv;
  const void* __restrict__ hcoef;
  const int* __restrict__ rchunk_handle;
  const int* __restrict__ rchunk_beg;
  const int* __restrict__ rchunk_ptr;
  int nrchunk;
  double* rpart;
  unsigned* rcount;
  // coarse
  int rc;
  const VT* __restrict__ W;
  const VT* __restrict__ WT;
  VT* c;
  VT* c2;
  // control
  double* part;            // [gridDim][4]
  PcgScalars* S;
  GridBarrier* bar;
  int iters;               // iterations to run in this launch (at most)
};

// y = H x for the rows of one 32-row slice, four lanes per row; tl in [0, 128)
template <typename VT, typename MT>
__device__ __forceinline__ void slice_rows(const PersistArgs<VT>& a, const MT* __restrict__ val, int slice, int tl,
                                           const Vec4<VT>* __restrict__ x, VT (&y)[3]) {
  const int part = tl & 3;
  const int rl = tl >> 2;
  const int row = slice * 32 + rl;
  const int len = row < a.n ? a.row_len[row] : 0;
  const int64_t g0 = a.slice_ptr[slice];
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
  for (int k0 = part; k0 < len; k0 += 16) {
    int c[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 4 * u;
      ok[u] = k < len;
      c[u] = ok[u] ? __ldg(a.col + (g0 + k) * 32 + rl) : 0;
    }
    Vec4<VT> xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = ok[u] ? ldv(x + c[u]) : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (!ok[u]) continue;
      const MT* v = val + (g0 + k0 + 4 * u) * 288 + rl;
      y0 += load_as<VT>(v[0]) * xv[u].x + load_as<VT>(v[32]) * xv[u].y + load_as<VT>(v[64]) * xv[u].z;
      y1 += load_as<VT>(v[96]) * xv[u].x + load_as<VT>(v[128]) * xv[u].y + load_as<VT>(v[160]) * xv[u].z;
      y2 += load_as<VT>(v[192]) * xv[u].x + load_as<VT>(v[224]) * xv[u].y + load_as<VT>(v[256]) * xv[u].z;
    }
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

template <typename VT>
__device__ __forceinline__ Vec4<VT> dinv_mul(const VT* __restrict__ dinv, int row, const Vec4<VT>& r, VT w) {
  const VT* D = dinv + (int64_t)row * 9;
  return Vec4<VT>{w * (D[0] * r.x + D[1] * r.y + D[2] * r.z), w * (D[3] * r.x + D[4] * r.y + D[5] * r.z),
                  w * (D[6] * r.x + D[7] * r.y + D[8] * r.z), VT(0)};
}

// sum of slot k of all blocks' partials, in block order (identical in every block)
__device__ __forceinline__ double total_of(const double* part, unsigned nblocks, int k) {
  __shared__ double tot;
  __syncthreads();
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)nblocks; b += 32) s += __ldcg(part + (size_t)b * 4 + k);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) tot = s;
  }
  __syncthreads();
  return tot;
}

// CYCLE: 0 block Jacobi, 1 additive two-level, 2 multiplicative two-level.
// The PCG scalars live in registers of every block (identical everywhere,
// since every block reduces the same partials in the same order); S is read
// at entry and written back by block 0 at exit.
template <typename VT, typename MT, int CYCLE>
__global__ void __launch_bounds__(kPersistThreads) k_pcg_persistent(PersistArgs<VT> a, const MT* __restrict__ val) {
  const unsigned nb = gridDim.x;
  const int tid = threadIdx.x;
  const int tl = tid & 127;
  const int sub = tid >> 7;
  const int gthreads = nb * kPersistThreads;
  const int gtid = blockIdx.x * kPersistThreads + tid;
  PcgScalars* S = a.S;
  double rz = S->rz, beta = S->beta, rr = S->rr, alpha = S->alpha, pqv = S->pq;
  const double tol2 = S->tol2;
  int iter = S->iter, done = S->done;
  const int max_iter = S->max_iter;
  bool ok = true;
  for (int it = 0; it < a.iters && !done; ++it) {
    // ---- A: product of the preconditioned residual, direction update, p.q
    {
      const VT vb = (VT)beta;
      double acc[1] = {0.0};
      for (int slice = blockIdx.x * 2 + sub; slice < a.n_slices; slice += nb * 2) {
        VT w[3];
        slice_rows<VT, MT>(a, val, slice, tl, a.zf, w);
        const int row = slice * 32 + (tl >> 2);
        if ((tl & 3) == 0 && row < a.n) {
          const Vec4<VT> zv = ldv(a.zf + row), pv = ldv(a.p + row), qv = ldv(a.q + row);
          const Vec4<VT> pn{zv.x + vb * pv.x, zv.y + vb * pv.y, zv.z + vb * pv.z, VT(0)};
          const Vec4<VT> qn{w[0] + vb * qv.x, w[1] + vb * qv.y, w[2] + vb * qv.z, VT(0)};
          a.p[row] = pn;
          a.q[row] = qn;
          acc[0] += (double)pn.x * qn.x + (double)pn.y * qn.y + (double)pn.z * qn.z;
        }
      }
      block_sum_p<1>(acc);
      if (tid == 0) a.part[(size_t)blockIdx.x * 4] = acc[0];
    }
    if (!(ok = grid_barrier(a.bar, nb))) break;
    pqv = total_of(a.part, nb, 0);
    if (!(pqv > 0.0) || !isfinite(pqv)) { done = 3; break; }
    alpha = rz / pqv;
    // ---- B: x, r update; smoothing term (or block-Jacobi z); |r|^2 (and r.z)
    {
      const VT va = (VT)alpha;
      double acc[2] = {0.0, 0.0};
      for (int row = gtid; row < a.n; row += gthreads) {
        const Vec4<VT> pv = ldv(a.p + row), qv = ldv(a.q + row);
        Vec4<VT> xv = ldv(a.x + row), rv = ldv(a.r + row);
        xv.x += va * pv.x; xv.y += va * pv.y; xv.z += va * pv.z;
        rv.x -= va * qv.x; rv.y -= va * qv.y; rv.z -= va * qv.z;
        a.x[row] = xv;
        a.r[row] = rv;
        acc[0] += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
        if (CYCLE == 0) {
          const Vec4<VT> zv = dinv_mul<VT>(a.dinv, row, rv, VT(1));
          a.zf[row] = zv;
          acc[1] += (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
        } else {
          a.z1[row] = dinv_mul<VT>(a.dinv, row, rv, a.omega);
        }
      }
      block_sum_p<2>(acc);
      if (tid == 0) { a.part[(size_t)blockIdx.x * 4 + 1] = acc[0]; a.part[(size_t)blockIdx.x * 4 + 2] = acc[1]; }
    }
    if (!(ok = grid_barrier(a.bar, nb))) break;
    rr = total_of(a.part, nb, 1);
    ++iter;
    if (!isfinite(rr)) { done = 3; break; }
    if (rr <= tol2) { done = 1; break; }
    if (iter >= max_iter) { done = 2; break; }
    if (CYCLE == 0) {
      const double rz_new = total_of(a.part, nb, 2);
      if (!(rz_new > 0.0) || !isfinite(rz_new)) { done = 3; break; }
      beta = rz_new / rz;
      rz = rz_new;
      continue;
    }
    // ---- C (multiplicative): t = r - H z1
    const Vec4<VT>* rsrc = a.r;
    if (CYCLE == 2) {
      for (int slice = blockIdx.x * 2 + sub; slice < a.n_slices; slice += nb * 2) {
        VT w[3];
        slice_rows<VT, MT>(a, val, slice, tl, a.z1, w);
        const int row = slice * 32 + (tl >> 2);
        if ((tl & 3) == 0 && row < a.n) {
          const Vec4<VT> rv = ldv(a.r + row);
          a.t[row] = Vec4<VT>{rv.x - w[0], rv.y - w[1], rv.z - w[2], VT(0)};
        }
      }
      rsrc = a.t;
      if (!(ok = grid_barrier(a.bar, nb))) break;
    }
    // ---- D: restriction; the last chunk of a handle to finish writes c_j
    for (int ch = blockIdx.x; ch < a.nrchunk; ch += nb) {
      const int j = a.rchunk_handle[ch];
      const int pidx = a.rchunk_beg[ch] + tid;
      VT acc[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[k] = VT(0);
      if (pidx < a.hrow[j + 1]) {
        const Vec4<VT> cf = ((const Vec4<VT>*)a.hcoef)[pidx];
        const Vec4<VT> rv = ldv(rsrc + a.hv[pidx]);
        const VT rcv[3] = {rv.x, rv.y, rv.z};
        const VT av[4] = {cf.x, cf.y, cf.z, cf.w};
#pragma unroll
        for (int cc = 0; cc < 3; ++cc)
#pragma unroll
          for (int l = 0; l < 4; ++l) acc[4 * cc + l] = rcv[cc] * av[l];
      }
      __shared__ VT shr[12][kPersistThreads / 32];
      __shared__ bool last;
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        VT sv = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sv += __shfl_xor_sync(0xffffffffu, sv, o);
        if (lane == 0) shr[k][warp] = sv;
      }
      __syncthreads();
      if (tid < 12) {
        VT sv = VT(0);
        for (int w = 0; w < kPersistThreads / 32; ++w) sv += shr[tid][w];
        a.rpart[12 * (int64_t)ch + tid] = (double)sv;
      }
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const unsigned nch = (unsigned)(a.rchunk_ptr[j + 1] - a.rchunk_ptr[j]);
        last = (atomicAdd(a.rcount + j, 1u) == nch - 1);
      }
      __syncthreads();
      if (last) {
        __threadfence();
        if (tid < 12) {
          const double sv = ordered_sum_ldcg(a.rpart + tid, 12, a.rchunk_ptr[j], a.rchunk_ptr[j + 1]);
          a.c[12 * (int64_t)j + tid] = (VT)sv;
        }
        if (tid == 0) a.rcount[j] = 0;
      }
      __syncthreads();
    }
    if (!(ok = grid_barrier(a.bar, nb))) break;
    // ---- F, G: c2 = W c (lower), c = W^T c2 (upper); one warp per row
    {
      constexpr int EV = 16 / sizeof(VT);
      using V16 = typename std::conditional<sizeof(VT) == 4, float4, double2>::type;
      const int lane = tid & 31;
      const int gw = gtid >> 5, nw = gthreads >> 5;
      for (int pass = 0; pass < 2 && ok; ++pass) {
        const VT* Wm = pass == 0 ? a.W : a.WT;
        const VT* xin = pass == 0 ? a.c : a.c2;
        VT* yout = pass == 0 ? a.c2 : a.c;
        for (int row = gw; row < a.rc; row += nw) {
          const int v0 = pass == 0 ? 0 : row / EV;
          const int v1 = pass == 0 ? (row + EV) / EV : a.rc / EV;
          const V16* Wr = reinterpret_cast<const V16*>(Wm + (int64_t)row * a.rc);
          const V16* xv = reinterpret_cast<const V16*>(xin);
          VT acc = VT(0);
#pragma unroll 4
          for (int cidx = v0 + lane; cidx < v1; cidx += 32) {
            const V16 w = Wr[cidx];
            const V16 bv = __ldcg(xv + cidx);
            if constexpr (sizeof(VT) == 4) acc += w.x * bv.x + w.y * bv.y + w.z * bv.z + w.w * bv.w;
            else acc += w.x * bv.x + w.y * bv.y;
          }
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (lane == 0) yout[row] = acc;
        }
        ok = grid_barrier(a.bar, nb);
      }
      if (!ok) break;
    }
    // ---- H: z1 += U c (additive: this is z, with r.z)
    {
      double acc[1] = {0.0};
      const Vec4<VT>* coef = (const Vec4<VT>*)a.vcoef;
      for (int v = gtid; v < a.n; v += gthreads) {
        VT o0 = VT(0), o1 = VT(0), o2 = VT(0);
        for (int k = a.vrow[v]; k < a.vrow[v + 1]; ++k) {
          const Vec4<VT> cf = coef[k];
          const Vec4<VT>* qj = (const Vec4<VT>*)(a.c + 12 * (int64_t)a.vh[k]);
          const Vec4<VT> q0 = ldv(qj), q1 = ldv(qj + 1), q2 = ldv(qj + 2);
          o0 += cf.x * q0.x + cf.y * q0.y + cf.z * q0.z + cf.w * q0.w;
          o1 += cf.x * q1.x + cf.y * q1.y + cf.z * q1.z + cf.w * q1.w;
          o2 += cf.x * q2.x + cf.y * q2.y + cf.z * q2.z + cf.w * q2.w;
        }
        const Vec4<VT> zb = ldv(a.z1 + v);
        const Vec4<VT> zo{zb.x + o0, zb.y + o1, zb.z + o2, VT(0)};
        a.z1[v] = zo;
        if (CYCLE == 1) {
          const Vec4<VT> rv = ldv(a.r + v);
          acc[0] += (double)rv.x * zo.x + (double)rv.y * zo.y + (double)rv.z * zo.z;
        }
      }
      if (CYCLE == 1) {
        block_sum_p<1>(acc);
        if (tid == 0) a.part[(size_t)blockIdx.x * 4 + 3] = acc[0];
      }
    }
    if (!(ok = grid_barrier(a.bar, nb))) break;
    // ---- I (multiplicative): zf = z1 + omega D^{-1} (r - H z1), r.zf
    if (CYCLE == 2) {
      double acc[1] = {0.0};
      for (int slice = blockIdx.x * 2 + sub; slice < a.n_slices; slice += nb * 2) {
        VT w[3];
        slice_rows<VT, MT>(a, val, slice, tl, a.z1, w);
        const int row = slice * 32 + (tl >> 2);
        if ((tl & 3) == 0 && row < a.n) {
          const Vec4<VT> rv = ldv(a.r + row), zv = ldv(a.z1 + row);
          const Vec4<VT> tv{rv.x - w[0], rv.y - w[1], rv.z - w[2], VT(0)};
          const Vec4<VT> sv = dinv_mul<VT>(a.dinv, row, tv, a.omega);
          const Vec4<VT> zo{zv.x + sv.x, zv.y + sv.y, zv.z + sv.z, VT(0)};
          a.zf[row] = zo;
          acc[0] += (double)rv.x * zo.x + (double)rv.y * zo.y + (double)rv.z * zo.z;
        }
      }
      block_sum_p<1>(acc);
      if (tid == 0) a.part[(size_t)blockIdx.x * 4 + 3] = acc[0];
      if (!(ok = grid_barrier(a.bar, nb))) break;
    }
    const double rz_new = total_of(a.part, nb, 3);
    if (!(rz_new > 0.0) || !isfinite(rz_new)) { done = (rr <= tol2) ? 1 : 3; break; }
    beta = rz_new / rz;
    rz = rz_new;
  }
  if (blockIdx.x == 0 && tid == 0) {
    S->rz = rz; S->beta = beta; S->rr = rr; S->alpha = alpha; S->pq = pqv;
    S->iter = iter;
    S->done = ok ? done : 4;
  }
}

}  // namespace mls

using namespace mls;

namespace mls {

template <typename VT, typename MT>
static mls_status launch_persistent_t(mls_ctx* ctx, int cycle, int iters) {
  PersistArgs<VT> a;
  a.n = ctx->n;
  a.n_slices = ctx->n_slices;
  a.slice_ptr = ctx->slice_ptr;
  a.col = ctx->col;
  a.row_len = ctx->row_len;
  a.dinv = (const VT*)ctx->dinv;
  a.omega = (VT)ctx->omega_eff;
  a.x = (Vec4<VT>*)ctx->vx;
  a.r = (Vec4<VT>*)ctx->vr;
  a.p = (Vec4<VT>*)ctx->vp;
  a.q = (Vec4<VT>*)ctx->vq;
  a.z1 = (Vec4<VT>*)ctx->vz;
  a.zf = (cycle == 2) ? (Vec4<VT>*)ctx->vz2 : (Vec4<VT>*)ctx->vz;
  a.t = (Vec4<VT>*)ctx->vw;
  const Basis& B = ctx->basis;
  a.m = B.m;
  a.vrow = B.vrow; a.vh = B.vh; a.vcoef = B.vcoef;
  a.hrow = B.hrow; a.hv = B.hv; a.hcoef = B.hcoef;
  a.rchunk_handle = B.rchunk_handle; a.rchunk_beg = B.rchunk_beg; a.rchunk_ptr = B.rchunk_ptr;
  a.nrchunk = B.nrchunk; a.rpart = B.rpart; a.rcount = B.rcount;
  a.rc = 12 * B.m;
  a.W = (const VT*)ctx->Linv; a.WT = (const VT*)ctx->LinvT;
  a.c = (VT*)ctx->cvec; a.c2 = (VT*)ctx->cvec2;
  a.part = ctx->persist_part;
  a.S = ctx->pcg;
  a.bar = (GridBarrier*)ctx->persist_bar;
  a.iters = iters;
  const MT* val = (const MT*)ctx->hval;
  void* fn;
  switch (cycle) {
    case 0: fn = (void*)k_pcg_persistent<VT, MT, 0>; break;
    case 1: fn = (void*)k_pcg_persistent<VT, MT, 1>; break;
    default: fn = (void*)k_pcg_persistent<VT, MT, 2>; break;
  }
  // Grid size: every block must be resident at once (a cooperative launch
  // checks this).  Default 2 blocks per SM: enough warps to overlap the
  // gathers of the products, few enough arrivals to keep each grid barrier
  // short.
  const int key = ctx->opt.persist_blocks_per_sm * 64 + ctx->opt.precision * 8 + cycle;
  if (ctx->persist_blocks == 0 || ctx->persist_bps != key) {
    int occ = 0, nsm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kPersistThreads, 0) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      return fail(ctx, MLS_ECUDA, "persistent PCG: occupancy query failed");
    }
    const int want = ctx->opt.persist_blocks_per_sm > 0 ? ctx->opt.persist_blocks_per_sm : 2;
    ctx->persist_blocks = std::min(nsm * std::min(occ, want), kMaxPersistBlocks);
    ctx->persist_bps = key;
  }
  int nb = ctx->persist_blocks;
  void* args[] = {&a, (void*)&val};
  ++ctx->launches;
  cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(nb), dim3(kPersistThreads), args, 0, ctx->stream);
  return cuda_check(ctx, e, "persistent PCG launch");
}

// Self-test of the bounded wait: every block arrives once at a barrier that
// expects `expected` arrivals.  With expected > gridDim.x no release comes;
// each waiting block gives up after spin_limit polls (or once another block
// has flagged the error), counts itself in gave_up and returns, so the kernel
// always ends.
__global__ void k_barrier_probe(GridBarrier* bar, unsigned expected, unsigned spin_limit, int* gave_up) {
  const bool ok = grid_barrier(bar, expected, spin_limit);
  if (threadIdx.x == 0 && !ok) atomicAdd(gave_up, 1);
}

mls_status launch_persistent_pcg(mls_ctx* ctx, int cycle, int iters) {
  switch (ctx->opt.precision) {
    case MLS_FP64: return launch_persistent_t<double, double>(ctx, cycle, iters);
    case MLS_MIXED_FP32: return launch_persistent_t<float, float>(ctx, cycle, iters);
    default: return launch_persistent_t<float, __nv_bfloat16>(ctx, cycle, iters);
  }
}

}  // namespace mls

extern "C" mls_status mls_selftest_barrier(int32_t blocks, int32_t expected, int32_t spin_limit, int32_t* gave_up,
                                           void* stream) {
  if (!gave_up || blocks < 1 || expected < 1 || spin_limit < 1) return MLS_EINVAL;
  *gave_up = 0;
  cudaStream_t s = (cudaStream_t)stream;
  void* mem = nullptr;
  if (cudaMalloc(&mem, 128) != cudaSuccess) { cudaGetLastError(); return MLS_ENOMEM; }
  GridBarrier* bar = (GridBarrier*)mem;
  int* count = (int*)((char*)mem + 64);
  mls_status st = MLS_OK;
  if (cudaMemsetAsync(mem, 0, 128, s) != cudaSuccess) st = MLS_ECUDA;
  unsigned ex = (unsigned)expected, sl = (unsigned)spin_limit;
  void* args[] = {&bar, &ex, &sl, &count};
  if (st == MLS_OK &&
      cudaLaunchCooperativeKernel((void*)k_barrier_probe, dim3(blocks), dim3(kPersistThreads), args, 0, s) != cudaSuccess)
    st = MLS_ECUDA;   // e.g. more blocks than can be co-resident
  int host = 0;
  if (st == MLS_OK && (cudaMemcpyAsync(&host, count, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                       cudaStreamSynchronize(s) != cudaSuccess))
    st = MLS_ECUDA;
  cudaGetLastError();
  cudaFree(mem);
  if (st != MLS_OK) return st;
  *gave_up = host;
  return host > 0 ? MLS_ETIMEOUT : MLS_OK;
}
