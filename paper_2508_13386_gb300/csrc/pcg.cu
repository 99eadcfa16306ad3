// Sparse matrix-vector product with the SELL-32 block matrix H and the
// preconditioned conjugate gradient loop on it (the Newton linear solve
// H d = -g of Eq. 5, preconditioned as in Sec. 3.7).
//
// PCG runs entirely on the device: the dot products p.q, r.r and r.z are
// order-independent fixed-point sums that every block adds to with
// fire-and-forget atomics, and the kernel that needs alpha or beta rebuilds it
// from the sum (one thread per block), so one iteration is two (block
// Jacobi) or more (two-level) kernel launches with no host round trip and no
// arrival counter.  The direction update p = z + beta p is folded into the
// product kernel through q = H p = H z + beta q_old, so the kernel that reads
// neighbours (the product) needs only z, which is complete when it starts.
// Dot products and norms accumulate in float64 in every precision mode.
#include "mls_internal.cuh"

namespace mls {

struct SellView {
  int n;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ col;
  const int* __restrict__ row_len;
};

template <typename VT, typename MT>
__device__ __forceinline__ void spmv_row(const SellView& A, const MT* __restrict__ val, int row,
                                         const Vec4<VT>* __restrict__ x, VT (&y)[3]) {
  const int slice = row >> 5, lane = row & 31;
  const int g0 = A.slice_ptr[slice];
  const int len = A.row_len[row];
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
  for (int k = 0; k < len; ++k) {
    const int64_t g = g0 + k;
    const int c = A.col[g * 32 + lane];
    const Vec4<VT> xv = x[c];
    const MT* v = val + g * 288 + lane;
    y0 += load_as<VT>(v[0]) * xv.x + load_as<VT>(v[32]) * xv.y + load_as<VT>(v[64]) * xv.z;
    y1 += load_as<VT>(v[96]) * xv.x + load_as<VT>(v[128]) * xv.y + load_as<VT>(v[160]) * xv.z;
    y2 += load_as<VT>(v[192]) * xv.x + load_as<VT>(v[224]) * xv.y + load_as<VT>(v[256]) * xv.z;
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

// One CTA of 128 threads per 32-row slice, four lanes per row (lane = 4 row + part):
// part p takes the slots k = p, p + 4, p + 8, ... of its row, so every load
// instruction of a warp covers 8 consecutive rows of 4 slot groups (four full
// 32-byte sectors); a lane first issues all its column indices and x gathers
// of a batch of up to four slots, then the values, to keep many loads in
// flight; the four partial rows are combined with two shuffles (no shared
// memory, no barrier).  Every lane returns the finished row in y.
constexpr int kSpmvWarps = 4;

template <typename VT, typename MT>
__device__ __forceinline__ void spmv_quad(const SellView& A, const MT* __restrict__ val, int slice,
                                          const Vec4<VT>* __restrict__ x, VT (&y)[3]) {
  const int part = threadIdx.x & 3;
  const int rl = threadIdx.x >> 2;        // row within the slice
  const int row = slice * 32 + rl;
  const int len = row < A.n ? A.row_len[row] : 0;
  const int64_t g0 = A.slice_ptr[slice];
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
  for (int k0 = part; k0 < len; k0 += 16) {
    int c[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 4 * u;
      ok[u] = k < len;
      c[u] = ok[u] ? __ldg(A.col + (g0 + k) * 32 + rl) : 0;
    }
    Vec4<VT> xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = ok[u] ? x[c[u]] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
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

// The same product split for chained launches: quad_load() reads the
// column indices and values of a lane's first slots (H does not change
// during a solve, so this may run before chain_wait(), while the previous
// kernel finishes); after the wait quad_gather() and quad_combine() below
// finish the rows.
// resident blocks of 128 threads per SM the row-quad kernels are compiled
// for: 12 in float32 (40 registers; measured 8% faster per product than 8
// blocks with four slots loaded ahead), 8 in float64 (wider values)
template <typename VT> constexpr int kQuadBlocks = sizeof(VT) == 4 ? 12 : 8;

template <typename VT>
struct QuadH {
  static constexpr int PF = 2;   // slots per lane loaded ahead (register budget, see kQuadBlocks)
  int len, rl, part;
  int64_t g0;
  int c[PF];
  VT w[PF][9];
};

template <typename VT, typename MT>
__device__ __forceinline__ void quad_load(const SellView& A, const MT* __restrict__ val, int slice, QuadH<VT>& h) {
  h.part = threadIdx.x & 3;
  h.rl = threadIdx.x >> 2;
  const int row = slice * 32 + h.rl;
  h.len = row < A.n ? A.row_len[row] : 0;
  h.g0 = A.slice_ptr[slice];
#pragma unroll
  for (int u = 0; u < QuadH<VT>::PF; ++u) {
    const int k = h.part + 4 * u;
    const bool ok = k < h.len;
    h.c[u] = ok ? __ldg(A.col + (h.g0 + k) * 32 + h.rl) : -1;
    const MT* v = val + (h.g0 + (ok ? k : 0)) * 288 + h.rl;
#pragma unroll
    for (int q = 0; q < 9; ++q) h.w[u][q] = ok ? load_as<VT>(v[32 * q]) : VT(0);
  }
}

// The rest of the product in two halves, so that a kernel can put other
// loads in flight between them: quad_gather() issues the x gathers of the
// slots that quad_load() holds; quad_combine() multiplies, adds the remaining
// slots (rows longer than 4 PF) and combines the four lanes of a row.
template <typename VT>
struct QuadX {
  Vec4<VT> x[QuadH<VT>::PF];
};

template <typename VT>
__device__ __forceinline__ void quad_gather(const QuadH<VT>& h, const Vec4<VT>* __restrict__ x, QuadX<VT>& g) {
#pragma unroll
  for (int u = 0; u < QuadH<VT>::PF; ++u)
    g.x[u] = h.c[u] >= 0 ? x[h.c[u]] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
}

template <typename VT, typename MT>
__device__ __forceinline__ void quad_combine(const SellView& A, const MT* __restrict__ val, const QuadH<VT>& h,
                                             const QuadX<VT>& g, const Vec4<VT>* __restrict__ x, VT (&y)[3]) {
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
#pragma unroll
  for (int u = 0; u < QuadH<VT>::PF; ++u) {
    const Vec4<VT>& xv = g.x[u];   // zero for the empty slots, whose weights are zero too
    y0 += h.w[u][0] * xv.x + h.w[u][1] * xv.y + h.w[u][2] * xv.z;
    y1 += h.w[u][3] * xv.x + h.w[u][4] * xv.y + h.w[u][5] * xv.z;
    y2 += h.w[u][6] * xv.x + h.w[u][7] * xv.y + h.w[u][8] * xv.z;
  }
  for (int k = h.part + 4 * QuadH<VT>::PF; k < h.len; k += 4) {
    const int c = __ldg(A.col + (h.g0 + k) * 32 + h.rl);
    const Vec4<VT> xv = x[c];
    const MT* v = val + (h.g0 + k) * 288 + h.rl;
    y0 += load_as<VT>(v[0]) * xv.x + load_as<VT>(v[32]) * xv.y + load_as<VT>(v[64]) * xv.z;
    y1 += load_as<VT>(v[96]) * xv.x + load_as<VT>(v[128]) * xv.y + load_as<VT>(v[160]) * xv.z;
    y2 += load_as<VT>(v[192]) * xv.x + load_as<VT>(v[224]) * xv.y + load_as<VT>(v[256]) * xv.z;
  }
#pragma unroll
  for (int o = 1; o <= 2; o <<= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  y[0] = y0; y[1] = y1; y[2] = y2;
}

// the row this thread finishes (part 0 of each quad), or -1
__device__ __forceinline__ int quad_row(int slice, int n) {
  if (threadIdx.x & 3) return -1;
  const int row = slice * 32 + (threadIdx.x >> 2);
  return row < n ? row : -1;
}

template <typename VT>
__device__ __forceinline__ Vec4<VT> dinv_apply(const VT* __restrict__ dinv, int row, const Vec4<VT>& r, VT omega) {
  const VT* D = dinv + (int64_t)row * 9;
  return Vec4<VT>{omega * (D[0] * r.x + D[1] * r.y + D[2] * r.z),
                  omega * (D[3] * r.x + D[4] * r.y + D[5] * r.z),
                  omega * (D[6] * r.x + D[7] * r.y + D[8] * r.z), VT(0)};
}

// ---- plain product / residual ---------------------------------------------------------
template <typename VT, typename MT>
__global__ void __launch_bounds__(32 * kSpmvWarps, 16) k_spmv(SellView A, const MT* __restrict__ val,
                                                          const Vec4<VT>* __restrict__ x, Vec4<VT>* __restrict__ y) {
  VT r[3];
  spmv_quad<VT, MT>(A, val, blockIdx.x, x, r);
  const int row = quad_row(blockIdx.x, A.n);
  if (row >= 0) y[row] = Vec4<VT>{r[0], r[1], r[2], VT(0)};
}

// out = b - H x
template <typename VT, typename MT>
__global__ void __launch_bounds__(32 * kSpmvWarps, kQuadBlocks<VT>) k_residual(SellView A, const MT* __restrict__ val,
                                                              const Vec4<VT>* __restrict__ b,
                                                              const Vec4<VT>* __restrict__ x,
                                                              Vec4<VT>* __restrict__ out,
                                                              const PcgScalars* __restrict__ S) {
  QuadH<VT> hq;
  quad_load<VT, MT>(A, val, blockIdx.x, hq);
  chain_wait();
  chain_release();
  // the gathers, b and the stop flag are loaded together; no barrier
  // follows, so each thread may act on its own read of the flag
  QuadX<VT> gx;
  quad_gather<VT>(hq, x, gx);
  const int row = quad_row(blockIdx.x, A.n);
  Vec4<VT> bb{};
  if (row >= 0) bb = b[row];
  const int done = S ? S->done : 0;
  VT r[3];
  quad_combine<VT, MT>(A, val, hq, gx, x, r);
  if (row < 0 || done) return;
  out[row] = Vec4<VT>{bb.x - r[0], bb.y - r[1], bb.z - r[2], VT(0)};
}

template <typename VT>
__global__ void __launch_bounds__(kBlock) k_jacobi(int n, const VT* __restrict__ dinv,
                                                   const Vec4<VT>* __restrict__ r, Vec4<VT>* __restrict__ z,
                                                   VT omega, const PcgScalars* __restrict__ S) {
  if (S && S->done) return;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  z[row] = dinv_apply<VT>(dinv, row, r[row], omega);
}

// ---- PCG --------------------------------------------------------------------------------
// init: x = 0, r = b, p = q = 0; with block Jacobi also z = D^{-1} b and r.z
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_pcg_init(int n, const Vec4<VT>* __restrict__ b, Vec4<VT>* __restrict__ x,
                                                     Vec4<VT>* __restrict__ r, Vec4<VT>* __restrict__ z,
                                                     Vec4<VT>* __restrict__ p, Vec4<VT>* __restrict__ q,
                                                     const VT* __restrict__ dinv, int jacobi, double rtol,
                                                     int max_iter, GridReduce gr, unsigned long long* __restrict__ fix,
                                                     PcgScalars* __restrict__ S) {
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x == 0)
    for (int w = threadIdx.x; w < kFixWords; w += blockDim.x) fix[w] = 0ull;
  double acc[2] = {0.0, 0.0};  // b.b, r.z
  if (row < n) {
    const Vec4<VT> bv = b[row];
    const Vec4<VT> zero{VT(0), VT(0), VT(0), VT(0)};
    x[row] = zero; p[row] = zero; q[row] = zero;
    r[row] = bv;
    acc[0] = (double)bv.x * bv.x + (double)bv.y * bv.y + (double)bv.z * bv.z;
    if (jacobi) {
      const Vec4<VT> zv = dinv_apply<VT>(dinv, row, bv, VT(1));
      z[row] = zv;
      acc[1] = (double)bv.x * zv.x + (double)bv.y * zv.y + (double)bv.z * zv.z;
    }
  }
  if (grid_sum<2>(acc, gr, RS_PCG_RZ) && threadIdx.x == 0) {
    S->bb = acc[0];
    S->rr = acc[0];
    S->rz = acc[1];
    S->rrv[0] = acc[0];
    S->rzv[0] = acc[1];
    S->beta = 0.0;
    S->alpha = 0.0;
    S->pq = 0.0;
    S->iter = 0;
    S->max_iter = max_iter;
    S->tol2 = rtol * rtol * acc[0];
    S->done = (acc[0] == 0.0) ? 1 : 0;
  }
}

// zout = z2 + omega D^{-1} (r - H z2) (the post-smoothing of the symmetric
// two-level cycle), fused with r.zout.  Inside the loop (first = 0, iteration
// it) r.zout goes to the order-independent sum that opens iteration it + 1;
// on the application before the loop (first = 1) a grid sum sets rz_0.
template <typename VT, typename MT>
__global__ void __launch_bounds__(32 * kSpmvWarps, kQuadBlocks<VT>) k_post_smooth_rz(SellView A, const MT* __restrict__ val,
                                                                    const Vec4<VT>* __restrict__ r,
                                                                    const Vec4<VT>* __restrict__ z2,
                                                                    const VT* __restrict__ dinv, VT omega,
                                                                    Vec4<VT>* __restrict__ zout, int first, int it,
                                                                    GridReduce gr, unsigned long long* __restrict__ fix,
                                                                    PcgScalars* __restrict__ S) {
  QuadH<VT> hq;
  quad_load<VT, MT>(A, val, blockIdx.x, hq);
  chain_wait();
  chain_release();
  // gathers, this row's r and z2 and the block's stop flag in flight together
  QuadX<VT> gx;
  quad_gather<VT>(hq, z2, gx);
  const int row = quad_row(blockIdx.x, A.n);
  Vec4<VT> rv{};
  if (row >= 0) rv = r[row];
  // a row's first slot is its diagonal block: the row's own z2 is gathered
  const Vec4<VT> zv = gx.x[0];
  __shared__ int s_done, s_e;
  if (threadIdx.x == 0) {
    const int d = __ldcg(&S->done);
    const double rzp = __ldcg(&S->rzv[it & 1]);
    s_done = d;
    s_e = fix_exponent(rzp);
  }
  __syncthreads();
  if (s_done) return;
  double acc[1] = {0.0};
  VT hz[3];
  quad_combine<VT, MT>(A, val, hq, gx, z2, hz);
  if (row >= 0) {
    const Vec4<VT> t{rv.x - hz[0], rv.y - hz[1], rv.z - hz[2], VT(0)};
    const Vec4<VT> s = dinv_apply<VT>(dinv, row, t, omega);
    const Vec4<VT> zo{zv.x + s.x, zv.y + s.y, zv.z + s.z, VT(0)};
    zout[row] = zo;
    acc[0] = (double)rv.x * zo.x + (double)rv.y * zo.y + (double)rv.z * zo.z;
  }
  if (!first) {
    __shared__ double sh[1][32];
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) fix_add(fix_slot(fix, FX_RZ, (it + 1) & 1), acc[0], s_e);
    return;
  }
  if (grid_sum<1>(acc, gr, RS_PCG_RZ) && threadIdx.x == 0) {
    S->beta = 0.0;
    S->rz = acc[0];
    S->rzv[0] = acc[0];
    if (!(acc[0] > 0.0) || !isfinite(acc[0])) S->done = (S->rr <= S->tol2) ? 1 : 3;
  }
}

// w = H z; p = z + beta p; q = w + beta q; p.q into the sum that k_pcg_update
// reads.  Opens iteration it: every block rebuilds rz_it, rr_it and beta_it
// from the sums of iteration it - 1 (the same words, so the same values) and
// stops on convergence, the iteration cap or breakdown; block 0 publishes
// them.
template <typename VT, typename MT>
__global__ void __launch_bounds__(32 * kSpmvWarps, kQuadBlocks<VT>) k_pcg_spmv(SellView A, const MT* __restrict__ val,
                                                              const Vec4<VT>* __restrict__ z, Vec4<VT>* __restrict__ p,
                                                              Vec4<VT>* __restrict__ q, int it,
                                                              unsigned long long* __restrict__ fix,
                                                              PcgScalars* __restrict__ S) {
  QuadH<VT> hq;
  quad_load<VT, MT>(A, val, blockIdx.x, hq);
  chain_wait();
  chain_release();
  // The x gathers and (thread 0) the stop flag and the sums that open the
  // iteration are loaded together, before the block's barrier.  Block 0 of
  // this kernel may set S->done while other blocks start: one thread reads it
  // and takes the decision for the whole block, so the block stays uniform.
  QuadX<VT> gx;
  quad_gather<VT>(hq, z, gx);
  const int row = quad_row(blockIdx.x, A.n);
  __shared__ VT s_beta;
  __shared__ int s_done, s_e;
  if (threadIdx.x == 0) {
    const int done0 = S->done;
    const PcgHeadRaw raw = pcg_head_load(fix, it);
    int done = done0;
    if (!done0) {
      const PcgHead<VT> h = pcg_head<VT>(S, raw, it);
      if (blockIdx.x == 0) pcg_head_publish<VT>(S, fix, it, h);
      s_beta = h.beta;
      s_e = fix_exponent(h.rz);
      done = h.done;
    }
    s_done = done;
  }
  __syncthreads();
  if (s_done) return;
  // a row's first slot is its diagonal block: the row's own z is gathered
  const Vec4<VT> zv = gx.x[0];
  VT w[3];
  quad_combine<VT, MT>(A, val, hq, gx, z, w);
  double acc[1] = {0.0};
  if (row >= 0) {
    const VT beta = s_beta;
    const Vec4<VT> pv = p[row], qv = q[row];
    const Vec4<VT> pn{zv.x + beta * pv.x, zv.y + beta * pv.y, zv.z + beta * pv.z, VT(0)};
    const Vec4<VT> qn{w[0] + beta * qv.x, w[1] + beta * qv.y, w[2] + beta * qv.z, VT(0)};
    p[row] = pn;
    q[row] = qn;
    acc[0] = (double)pn.x * qn.x + (double)pn.y * qn.y + (double)pn.z * qn.z;
  }
  __shared__ double sh[1][32];
  block_sum<1>(acc, sh);
  if (threadIdx.x == 0) fix_add(fix_slot(fix, FX_PQ, it & 1), acc[0], s_e);
}

// the opening decision of iteration it on its own (one thread), launched at
// the end of each chunk of iterations before the host reads the scalars
__global__ void k_pcg_check(int it, unsigned long long* __restrict__ fix, PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  const PcgOpen o = pcg_open_load_warp(fix, S, it);  // one warp
  if (threadIdx.x != 0 || o.done) return;
  pcg_head_publish<double>(S, fix, it, pcg_head_open<double>(o, it));
}

// x += alpha p; r -= alpha q; then by mode: 1 = block Jacobi z = D^{-1} r with
// r.z; 2 = the smoothing term z = omega D^{-1} r of a two-level cycle.  r.r
// (and r.z in mode 1) go to the sums that open iteration it + 1; alpha =
// rz_it / p.q from the sum of k_pcg_spmv.  Block 0 clears the RR and RZ slots
// that k_pcg_spmv consumed.  One row per thread in 128-thread blocks: twice
// the blocks of a 256-thread launch, to spread the rows over more SMs.
constexpr int kUpdBlock = 128;
template <typename VT>
__global__ void __launch_bounds__(kUpdBlock) k_pcg_update(int n, Vec4<VT>* __restrict__ x, Vec4<VT>* __restrict__ r,
                                                       Vec4<VT>* __restrict__ z, const Vec4<VT>* __restrict__ p,
                                                       const Vec4<VT>* __restrict__ q, const VT* __restrict__ dinv,
                                                       int jacobi, VT omega, int it,
                                                       unsigned long long* __restrict__ fix,
                                                       PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  Vec4<VT> pv{}, qv{}, xv{}, rv{};
  if (row < n) { pv = p[row]; qv = q[row]; xv = x[row]; rv = r[row]; }
  __shared__ VT s_alpha;
  __shared__ int s_go, s_erz, s_err;
  if (threadIdx.x < 32) {
    // lanes 0-4: the p.q slot, lane 5: the stop flag, lanes 6-7: rz_it and
    // rr_it (the scale estimates of the sums this kernel adds to), in one
    // round trip
    const int lane = threadIdx.x;
    const unsigned long long* pqs = fix_slot(fix, FX_PQ, it & 1);
    unsigned long long w = 0ull;
    if (lane < 5) w = __ldcg(pqs + lane * kFixStride);
    else if (lane == 5) w = (unsigned long long)(unsigned)__ldcg(&S->done);
    else if (lane == 6) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rzv[it & 1]));
    else if (lane == 7) w = (unsigned long long)__double_as_longlong(__ldcg(&S->rrv[it & 1]));
    FixRaw pqr;
#pragma unroll
    for (int k = 0; k < 5; ++k) pqr.w[k] = __shfl_sync(0xffffffffu, w, k);
    const int done0 = (int)__shfl_sync(0xffffffffu, w, 5);
    const double rz = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 6));
    const double rr = __longlong_as_double((long long)__shfl_sync(0xffffffffu, w, 7));
    if (threadIdx.x == 0) {
      int go = 0;
      VT alpha = VT(0);
      if (!done0) {  // block 0 may set it on breakdown: read once per block
        bool bad;
        const double pq = fix_value(pqr, fix_exponent(rz), bad);
        go = !bad && dbl_positive(pq);
        if (go) alpha = ratio<VT>(rz, pq);
        if (blockIdx.x == 0) {
          S->pq = pq;
          if (!go) S->done = 3;  // breakdown: H or the preconditioner is not positive definite
          fix_clear(fix_slot(fix, FX_RR, it & 1));
          fix_clear(fix_slot(fix, FX_RZ, it & 1));
        }
      }
      s_go = go;
      s_alpha = alpha;
      s_erz = fix_exponent(rz);
      s_err = fix_exponent(rr);
    }
  }
  __syncthreads();
  if (!s_go) return;
  double acc[2] = {0.0, 0.0};  // r.r, r.z
  if (row < n) {
    const VT alpha = s_alpha;
    xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z;
    rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z;
    x[row] = xv;
    r[row] = rv;
    acc[0] = (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
    if (jacobi == 1) {
      const Vec4<VT> zv = dinv_apply<VT>(dinv, row, rv, VT(1));
      z[row] = zv;
      acc[1] = (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
    } else if (jacobi == 2) {
      z[row] = dinv_apply<VT>(dinv, row, rv, omega);
    }
  }
  __shared__ double sh[2][32];
  block_sum<2>(acc, sh);
  if (threadIdx.x == 0) {
    fix_add(fix_slot(fix, FX_RR, (it + 1) & 1), acc[0], s_err);
    if (jacobi == 1) fix_add(fix_slot(fix, FX_RZ, (it + 1) & 1), acc[1], s_erz);
  }
}

// ---- launchers ---------------------------------------------------------------------------
static SellView sell_view(mls_ctx* ctx) { return SellView{ctx->n, ctx->slice_ptr, ctx->col, ctx->row_len}; }
static inline int nblk(int64_t n) { return (int)((n + kBlock - 1) / kBlock); }

template <typename VT, typename MT>
static void spmv_t(mls_ctx* ctx, const void* values, const void* x, void* y) {
  { ++ctx->launches; k_spmv<VT, MT><<<ctx->n_slices, 32 * kSpmvWarps, 0, ctx->stream>>>(sell_view(ctx), (const MT*)values,
                                                           (const Vec4<VT>*)x, (Vec4<VT>*)y); }
}

mls_status launch_spmv_values(mls_ctx* ctx, const void* values, const void* x, void* y) {
  switch (ctx->opt.precision) {
    case MLS_FP64: spmv_t<double, double>(ctx, values, x, y); break;
    case MLS_MIXED_FP32: spmv_t<float, float>(ctx, values, x, y); break;
    default: spmv_t<float, __nv_bfloat16>(ctx, values, x, y); break;
  }
  return cuda_check(ctx, cudaGetLastError(), "k_spmv");
}

mls_status launch_spmv(mls_ctx* ctx, const void* x, void* y) { return launch_spmv_values(ctx, ctx->hval, x, y); }

template <typename VT, typename MT>
mls_status launch_residual_t(mls_ctx* ctx, const void* b, const void* x, void* out, const PcgScalars* S) {
  ++ctx->launches;
  return cuda_check(ctx, launch_chained(k_residual<VT, MT>, dim3(ctx->n_slices), dim3(32 * kSpmvWarps), ctx->stream,
                                        sell_view(ctx), (const MT*)ctx->hval, (const Vec4<VT>*)b, (const Vec4<VT>*)x,
                                        (Vec4<VT>*)out, S), "k_residual");
}

mls_status launch_residual(mls_ctx* ctx, const void* b, const void* x, void* out, const PcgScalars* S) {
  switch (ctx->opt.precision) {
    case MLS_FP64: return launch_residual_t<double, double>(ctx, b, x, out, S);
    case MLS_MIXED_FP32: return launch_residual_t<float, float>(ctx, b, x, out, S);
    default: return launch_residual_t<float, __nv_bfloat16>(ctx, b, x, out, S);
  }
}

template <typename VT, typename MT>
static mls_status post_smooth_t(mls_ctx* ctx, const void* r, const void* z2, void* zout, int first, int it,
                                PcgScalars* S) {
  ++ctx->launches;
  return cuda_check(ctx, launch_chained(k_post_smooth_rz<VT, MT>, dim3(ctx->n_slices), dim3(32 * kSpmvWarps), ctx->stream,
                                        sell_view(ctx), (const MT*)ctx->hval, (const Vec4<VT>*)r, (const Vec4<VT>*)z2,
                                        (const VT*)ctx->dinv, (VT)ctx->omega_eff, (Vec4<VT>*)zout, first, it, ctx->red,
                                        ctx->pcg_fix, S),
                    "k_post_smooth_rz");
}

mls_status launch_post_smooth_rz(mls_ctx* ctx, const void* r, const void* z2, void* zout, int first, int it,
                                 PcgScalars* S) {
  switch (ctx->opt.precision) {
    case MLS_FP64: return post_smooth_t<double, double>(ctx, r, z2, zout, first, it, S);
    case MLS_MIXED_FP32: return post_smooth_t<float, float>(ctx, r, z2, zout, first, it, S);
    default: return post_smooth_t<float, __nv_bfloat16>(ctx, r, z2, zout, first, it, S);
  }
}

mls_status launch_jacobi(mls_ctx* ctx, const void* r, void* z, double omega, const PcgScalars* S) {
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_jacobi<double><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const double*)ctx->dinv,
                                                               (const Vec4d*)r, (Vec4d*)z, omega, S); }
  else
    { ++ctx->launches; k_jacobi<float><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const float*)ctx->dinv,
                                                              (const Vec4f*)r, (Vec4f*)z, (float)omega, S); }
  return cuda_check(ctx, cudaGetLastError(), "k_jacobi");
}

mls_status precond_apply_dev(mls_ctx* ctx, const void* r, void* z, const PcgScalars* S);
mls_status two_level_pcg_step(mls_ctx* ctx, const void* r, void* z1, void* zfinal, int first, int it, PcgScalars* S);

template <typename VT, typename MT>
static mls_status pcg_t(mls_ctx* ctx, double rtol, int max_iter, int* iters, double* rel_res) {
  const int n = ctx->n;
  const int nb = nblk(n);
  const int nb_upd = (n + kUpdBlock - 1) / kUpdBlock;
  if (nb_upd > kMaxPartials || ctx->n_slices > kMaxPartials)
    return fail(ctx, MLS_EINVAL, "mesh too large for one reduction grid");
  const bool jacobi = ctx->opt.preconditioner == MLS_PRECOND_BLOCK_JACOBI || ctx->coarse_fallback;
  if (!jacobi && !ctx->coarse_ready) return fail(ctx, MLS_EINVAL, "two-level preconditioner needs mls_build_coarse");
  auto* b = (const Vec4<VT>*)ctx->vb;
  auto* x = (Vec4<VT>*)ctx->vx;
  auto* r = (Vec4<VT>*)ctx->vr;
  auto* z = (Vec4<VT>*)ctx->vz;
  auto* p = (Vec4<VT>*)ctx->vp;
  auto* q = (Vec4<VT>*)ctx->vq;
  const VT* dinv = (const VT*)ctx->dinv;
  PcgScalars* S = ctx->pcg;
  SellView A = sell_view(ctx);
  const MT* val = (const MT*)ctx->hval;
  { ++ctx->launches; k_pcg_init<VT><<<nb, kBlock, 0, ctx->stream>>>(n, b, x, r, z, p, q, dinv, jacobi ? 1 : 0, rtol, max_iter,
                                                 ctx->red, ctx->pcg_fix, S); }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "k_pcg_init");
  if (st != MLS_OK) return st;
  // two-level: z1 (in vz) holds the smoothing term and then U-corrected
  // iterate; zf is the preconditioned residual the product kernel reads
  const bool mult = ctx->opt.cycle == MLS_CYCLE_MULTIPLICATIVE;
  Vec4<VT>* z1 = z;
  Vec4<VT>* zf = (!jacobi && mult) ? (Vec4<VT>*)ctx->vz2 : z;
  if (!jacobi) {
    if ((st = launch_jacobi(ctx, r, z1, ctx->omega_eff, S)) != MLS_OK) return st;
    if ((st = two_level_pcg_step(ctx, r, z1, zf, 1, 0, S)) != MLS_OK) return st;
  }
  if (ctx->opt.persistent) {
    const int cycle = jacobi ? 0 : (mult ? 2 : 1);
    int tk = prof_begin(ctx, MLS_PROF_PCG_FUSED);
    if ((st = launch_persistent_pcg(ctx, cycle, max_iter)) != MLS_OK) return st;
    prof_end(ctx, tk);
    st = cuda_check(ctx, cudaMemcpyAsync(ctx->pcg_host, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost, ctx->stream),
                    "pcg readback");
    if (st != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "pcg sync")) != MLS_OK) return st;
    prof_flush(ctx);
    if (ctx->pcg_host->done == 4) {
      cudaMemsetAsync(ctx->persist_bar, 0, 64, ctx->stream);
      return fail(ctx, MLS_ETIMEOUT, "persistent PCG: a grid barrier wait gave up");
    }
  }
  const int chunk = ctx->opt.pcg_check_every > 0 ? ctx->opt.pcg_check_every : 16;
  const VT omega = (VT)ctx->omega_eff;
  int it = 0;  // iteration index; its parity selects the sums' slots
  for (; !ctx->opt.persistent;) {
    for (int c = 0; c < chunk; ++c, ++it) {
      int tk = prof_begin(ctx, MLS_PROF_SPMV);
      ++ctx->launches;
      if ((st = cuda_check(ctx, launch_chained(k_pcg_spmv<VT, MT>, dim3(ctx->n_slices), dim3(32 * kSpmvWarps), ctx->stream,
                                               A, val, (const Vec4<VT>*)zf, p, q, it, ctx->pcg_fix, S),
                           "k_pcg_spmv")) != MLS_OK)
        return st;
      prof_end(ctx, tk);
      tk = prof_begin(ctx, MLS_PROF_PCG_UPDATE);
      ++ctx->launches;
      if ((st = cuda_check(ctx, launch_chained(k_pcg_update<VT>, dim3(nb_upd), dim3(kUpdBlock), ctx->stream, n, x, r, z1,
                                               (const Vec4<VT>*)p, (const Vec4<VT>*)q, dinv, jacobi ? 1 : 2, omega,
                                               it, ctx->pcg_fix, S), "k_pcg_update")) != MLS_OK)
        return st;
      prof_end(ctx, tk);
      if (!jacobi) {
        tk = prof_begin(ctx, MLS_PROF_PRECOND);
        if ((st = two_level_pcg_step(ctx, r, z1, zf, 0, it, S)) != MLS_OK) return st;
        prof_end(ctx, tk);
      }
    }
    // the decision that opens the next iteration, before the host reads it
    ++ctx->launches;
    if ((st = cuda_check(ctx, launch_chained(k_pcg_check, dim3(1), dim3(32), ctx->stream, it, ctx->pcg_fix, S),
                         "k_pcg_check")) != MLS_OK)
      return st;
    st = cuda_check(ctx, cudaGetLastError(), "pcg iteration");
    if (st != MLS_OK) return st;
    st = cuda_check(ctx, cudaMemcpyAsync(ctx->pcg_host, S, sizeof(PcgScalars), cudaMemcpyDeviceToHost,
                                         ctx->stream), "pcg readback");
    if (st != MLS_OK) return st;
    st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "pcg sync");
    if (st != MLS_OK) return st;
    prof_flush(ctx);
    if (ctx->pcg_host->done) break;
  }
  const PcgScalars& h = *ctx->pcg_host;
  if (iters) *iters = h.iter;
  if (rel_res) *rel_res = h.bb > 0 ? sqrt(h.rr / h.bb) : 0.0;
  if (h.done == 3) return fail(ctx, MLS_ENONFINITE, "PCG breakdown (non-positive curvature or non-finite value)");
  if (h.done == 2) return fail(ctx, MLS_ENOTCONV, "PCG reached its iteration cap");
  return MLS_OK;
}

mls_status pcg_solve(mls_ctx* ctx, double rtol, int max_iter, int* iters, double* rel_res) {
  switch (ctx->opt.precision) {
    case MLS_FP64: return pcg_t<double, double>(ctx, rtol, max_iter, iters, rel_res);
    case MLS_MIXED_FP32: return pcg_t<float, float>(ctx, rtol, max_iter, iters, rel_res);
    default: return pcg_t<float, __nv_bfloat16>(ctx, rtol, max_iter, iters, rel_res);
  }
}

mls_status precond_apply(mls_ctx* ctx, const void* r, void* z) { return precond_apply_dev(ctx, r, z, nullptr); }

}  // namespace mls
