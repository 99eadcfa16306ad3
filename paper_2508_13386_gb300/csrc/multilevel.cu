// The two-level preconditioner built from the sparse LBS basis.
//
// Basis (Eq. LBS, Sec. 3.4-3.5): U[3v + c, 12j + 4c + l] = phi_j(v) a_l with
// a = [1, X_v - o_j].  Prolongation w = U q and restriction z = U^T r apply it
// without assembling U (the paper's CSR-like basis products, Sec. 3.7.1).
//
// Coarse operator: A_c = U^T H U (the subspace "sandwich" matrix of Alg. 2),
// formed explicitly in two sparse passes:
//   Y = H U       one thread per (row v, handle j reachable from v): the 3x12
//                 block Y_vj = sum_w H_vw phi_j(w) (I_3 (x) a_wj^T)
//   A_c = U^T Y   one CTA per coarse block row i: for each neighbour handle j,
//                 A_ij = sum_{v in supp i} phi_i(v) a_vi (x) Y_vj, summed in a
//                 fixed order (no atomics)
// then factored A_c = L L^T by a blocked right-looking Cholesky in float64,
// and inverted, W = L^{-1}, so that each coarse solve A_c^{-1} c = W^T (W c)
// is two dense triangular matrix-vector products spread over all SMs.
//
// Preconditioner (S = omega D^{-1}, D the 3x3 block diagonal of H,
// Q = U A_c^{-1} U^T):
//   additive        z = S r + Q r
//   multiplicative  z1 = S r; z2 = z1 + Q (r - H z1); z = z2 + S (r - H z2)
#include "mls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <type_traits>

namespace mls {

mls_status launch_residual(mls_ctx* ctx, const void* b, const void* x, void* out, const PcgScalars* S);
mls_status launch_jacobi(mls_ctx* ctx, const void* r, void* z, double omega, const PcgScalars* S);

static inline int nblk(int64_t n, int b = kBlock) { return (int)((n + b - 1) / b); }

// ---- host: basis upload and symbolic structure ---------------------------------------
mls_status basis_upload(mls_ctx* ctx, int m, const double* origins, const int* vrow, const int* handle,
                        const double* phi) {
  const int n = ctx->n;
  Basis& B = ctx->basis;
  if (m < 1) return fail(ctx, MLS_EINVAL, "n_handles must be >= 1");
  if (vrow[0] != 0) return fail(ctx, MLS_EINVAL, "vrow[0] must be 0");
  for (int v = 0; v < n; ++v)
    if (vrow[v + 1] < vrow[v]) return fail(ctx, MLS_EINVAL, "vrow must be non-decreasing");
  const int nnz = vrow[n];
  for (int k = 0; k < nnz; ++k)
    if (handle[k] < 0 || handle[k] >= m) return fail(ctx, MLS_EINVAL, "basis handle index out of range");
  // per-vertex lists sorted by handle, duplicates merged
  std::vector<int> h_vrow(n + 1, 0), h_vh;
  std::vector<double> h_vphi;
  h_vh.reserve(nnz);
  h_vphi.reserve(nnz);
  int maxk = 0;
  for (int v = 0; v < n; ++v) {
    std::vector<std::pair<int, double>> e;
    for (int k = vrow[v]; k < vrow[v + 1]; ++k) e.emplace_back(handle[k], phi[k]);
    std::sort(e.begin(), e.end());
    int cnt = 0;
    for (size_t q = 0; q < e.size(); ++q) {
      if (q > 0 && e[q].first == e[q - 1].first) { h_vphi.back() += e[q].second; continue; }
      h_vh.push_back(e[q].first);
      h_vphi.push_back(e[q].second);
      ++cnt;
    }
    h_vrow[v + 1] = h_vrow[v] + cnt;
    maxk = std::max(maxk, cnt);
  }
  const int nz = h_vrow[n];
  // transpose: per-handle vertex lists
  std::vector<int> h_hrow(m + 1, 0), h_hv(nz);
  std::vector<double> h_hphi(nz);
  for (int k = 0; k < nz; ++k) h_hrow[h_vh[k] + 1]++;
  for (int j = 0; j < m; ++j) h_hrow[j + 1] += h_hrow[j];
  {
    std::vector<int> fill(h_hrow.begin(), h_hrow.end() - 1);
    for (int v = 0; v < n; ++v)
      for (int k = h_vrow[v]; k < h_vrow[v + 1]; ++k) {
        const int p = fill[h_vh[k]]++;
        h_hv[p] = v;
        h_hphi[p] = h_vphi[k];
      }
  }
  // K_v: handles reachable from row v through the sparsity of H
  const std::vector<int>& sp = ctx->h_slice_ptr;
  const std::vector<int>& rl = ctx->h_row_len;
  const std::vector<int>& hc = ctx->h_col;
  auto col_of = [&](int v, int k) { return hc[((size_t)sp[v >> 5] + k) * 32 + (v & 31)]; };
  std::vector<int> h_yrow(n + 1, 0), h_yh;
  std::vector<int16_t> h_yslot((size_t)ctx->n_groups * 32 * std::max(maxk, 1), (int16_t)-1);
  std::vector<int> mark(m, -1), local(m, 0);
  for (int v = 0; v < n; ++v) {
    std::vector<int> Kv;
    for (int k = 0; k < rl[v]; ++k) {
      const int w = col_of(v, k);
      for (int q = h_vrow[w]; q < h_vrow[w + 1]; ++q) {
        const int j = h_vh[q];
        if (mark[j] != v) { mark[j] = v; Kv.push_back(j); }
      }
    }
    std::sort(Kv.begin(), Kv.end());
    for (size_t q = 0; q < Kv.size(); ++q) local[Kv[q]] = (int)q;
    for (int k = 0; k < rl[v]; ++k) {
      const int w = col_of(v, k);
      const size_t slot = ((size_t)sp[v >> 5] + k) * 32 + (v & 31);
      for (int q = h_vrow[w]; q < h_vrow[w + 1]; ++q)
        h_yslot[slot * maxk + (q - h_vrow[w])] = (int16_t)local[h_vh[q]];
    }
    h_yrow[v + 1] = h_yrow[v] + (int)Kv.size();
    h_yh.insert(h_yh.end(), Kv.begin(), Kv.end());
    B.maxkv = std::max(B.maxkv, (int)Kv.size());
  }
  const int64_t ny = h_yrow[n];
  // coarse block-row neighbours N_i = union of K_v over v in supp(i), and the
  // per-(i, j) entry lists (v, y index) sorted by neighbour slot
  std::vector<int> h_hn_row(m + 1, 0), h_hn;
  std::vector<int> h_ent_ptr(1, 0), h_ent_y, h_ent_v;
  std::vector<double> h_ent_phi;
  std::vector<int> mark2(m, -1);
  std::vector<std::vector<std::pair<int, int>>> per_slot;  // reused
  for (int i = 0; i < m; ++i) {
    std::vector<int> Ni;
    for (int p = h_hrow[i]; p < h_hrow[i + 1]; ++p) {
      const int v = h_hv[p];
      for (int q = h_yrow[v]; q < h_yrow[v + 1]; ++q) {
        const int j = h_yh[q];
        if (mark2[j] != i) { mark2[j] = i; Ni.push_back(j); }
      }
    }
    std::sort(Ni.begin(), Ni.end());
    for (size_t q = 0; q < Ni.size(); ++q) local[Ni[q]] = (int)q;
    per_slot.assign(Ni.size(), {});
    for (int p = h_hrow[i]; p < h_hrow[i + 1]; ++p) {
      const int v = h_hv[p];
      for (int q = h_yrow[v]; q < h_yrow[v + 1]; ++q) per_slot[local[h_yh[q]]].emplace_back(p, q);
    }
    for (size_t s = 0; s < Ni.size(); ++s) {
      for (auto& pq : per_slot[s]) {
        h_ent_y.push_back(pq.second);
        h_ent_v.push_back(h_hv[pq.first]);
        h_ent_phi.push_back(h_hphi[pq.first]);
      }
      h_ent_ptr.push_back((int)h_ent_y.size());
    }
    h_hn_row[i + 1] = h_hn_row[i] + (int)Ni.size();
    h_hn.insert(h_hn.end(), Ni.begin(), Ni.end());
  }
  const int nbk = h_hn_row[m];
  const size_t nent = h_ent_y.size();
  // per-entry coefficients (phi, phi a) in solve precision, vertex- and
  // handle-major; restriction chunks of at most kRestrictChunk entries
  const bool fp64 = ctx->opt.precision == MLS_FP64;
  std::vector<double> h_vcoef(4 * (size_t)nz), h_hcoef(4 * (size_t)nz);
  for (int v = 0; v < n; ++v)
    for (int k = h_vrow[v]; k < h_vrow[v + 1]; ++k) {
      const int j = h_vh[k];
      const double ph = h_vphi[k];
      h_vcoef[4 * (size_t)k + 0] = ph;
      for (int c = 0; c < 3; ++c) h_vcoef[4 * (size_t)k + 1 + c] = ph * (ctx->h_X[3 * (size_t)v + c] - origins[3 * j + c]);
    }
  for (int j = 0; j < m; ++j)
    for (int p = h_hrow[j]; p < h_hrow[j + 1]; ++p) {
      const int v = h_hv[p];
      const double ph = h_hphi[p];
      h_hcoef[4 * (size_t)p + 0] = ph;
      for (int c = 0; c < 3; ++c) h_hcoef[4 * (size_t)p + 1 + c] = ph * (ctx->h_X[3 * (size_t)v + c] - origins[3 * j + c]);
    }
  std::vector<int> h_rchunk_handle, h_rchunk_beg;
  std::vector<int> h_rchunk_ptr(m + 1, 0);
  for (int j = 0; j < m; ++j) {
    for (int b = h_hrow[j]; b < h_hrow[j + 1]; b += kRestrictChunk) {
      h_rchunk_handle.push_back(j);
      h_rchunk_beg.push_back(b);
    }
    if (h_hrow[j + 1] == h_hrow[j]) {  // empty handle: one empty chunk writes its zeros
      h_rchunk_handle.push_back(j);
      h_rchunk_beg.push_back(h_hrow[j]);
    }
    h_rchunk_ptr[j + 1] = (int)h_rchunk_handle.size();
  }
  const int nrchunk = (int)h_rchunk_handle.size();
  // chunks of at most kGalerkinChunk entries that never cross a coarse block
  std::vector<int> h_chunk_ptr(1, 0), h_chunk_beg, h_slot_row(nbk);
  for (int i = 0; i < m; ++i)
    for (int sl = h_hn_row[i]; sl < h_hn_row[i + 1]; ++sl) h_slot_row[sl] = i;
  for (int sl = 0; sl < nbk; ++sl) {
    for (int b = h_ent_ptr[sl]; b < h_ent_ptr[sl + 1]; b += kGalerkinChunk) h_chunk_beg.push_back(b);
    h_chunk_ptr.push_back((int)h_chunk_beg.size());
  }
  const int nchunk = (int)h_chunk_beg.size();

  // device copies
  auto up = [&](void** dst, const void* src, size_t bytes) -> mls_status {
    mls_status st = dalloc(ctx, dst, std::max<size_t>(bytes, 16));
    if (st != MLS_OK) return st;
    if (bytes) return cuda_check(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "basis upload");
    return MLS_OK;
  };
  mls_status st;
  if ((st = up((void**)&B.vrow, h_vrow.data(), sizeof(int) * (n + 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.vh, h_vh.data(), sizeof(int) * nz)) != MLS_OK) return st;
  if ((st = up((void**)&B.vphi, h_vphi.data(), sizeof(double) * nz)) != MLS_OK) return st;
  if ((st = up((void**)&B.hrow, h_hrow.data(), sizeof(int) * (m + 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.hv, h_hv.data(), sizeof(int) * nz)) != MLS_OK) return st;
  if ((st = up((void**)&B.hphi, h_hphi.data(), sizeof(double) * nz)) != MLS_OK) return st;
  if ((st = up((void**)&B.origins, origins, sizeof(double) * 3 * m)) != MLS_OK) return st;
  if ((st = up((void**)&B.yrow, h_yrow.data(), sizeof(int) * (n + 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.yh, h_yh.data(), sizeof(int) * ny)) != MLS_OK) return st;
  if ((st = up((void**)&B.yslot, h_yslot.data(), sizeof(int16_t) * h_yslot.size())) != MLS_OK) return st;
  if ((st = up((void**)&B.hn_row, h_hn_row.data(), sizeof(int) * (m + 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.hn, h_hn.data(), sizeof(int) * nbk)) != MLS_OK) return st;
  if ((st = up((void**)&B.ent_ptr, h_ent_ptr.data(), sizeof(int) * (nbk + 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.ent_y, h_ent_y.data(), sizeof(int) * nent)) != MLS_OK) return st;
  if ((st = up((void**)&B.ent_v, h_ent_v.data(), sizeof(int) * nent)) != MLS_OK) return st;
  if ((st = up((void**)&B.ent_phi, h_ent_phi.data(), sizeof(double) * nent)) != MLS_OK) return st;
  if ((st = up((void**)&B.chunk_ptr, h_chunk_ptr.data(), sizeof(int) * (nbk + 1))) != MLS_OK) return st;
  if (fp64) {
    if ((st = up(&B.vcoef, h_vcoef.data(), sizeof(double) * h_vcoef.size())) != MLS_OK) return st;
    if ((st = up(&B.hcoef, h_hcoef.data(), sizeof(double) * h_hcoef.size())) != MLS_OK) return st;
  } else {
    std::vector<float> fv(h_vcoef.begin(), h_vcoef.end()), fh(h_hcoef.begin(), h_hcoef.end());
    if ((st = up(&B.vcoef, fv.data(), sizeof(float) * fv.size())) != MLS_OK) return st;
    if ((st = up(&B.hcoef, fh.data(), sizeof(float) * fh.size())) != MLS_OK) return st;
  }
  if ((st = up((void**)&B.rchunk_handle, h_rchunk_handle.data(), sizeof(int) * nrchunk)) != MLS_OK) return st;
  if ((st = up((void**)&B.rchunk_beg, h_rchunk_beg.data(), sizeof(int) * nrchunk)) != MLS_OK) return st;
  if ((st = up((void**)&B.rchunk_ptr, h_rchunk_ptr.data(), sizeof(int) * (m + 1))) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&B.rpart, sizeof(double) * 12 * nrchunk)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&B.rcount, sizeof(unsigned) * m)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemset(B.rcount, 0, sizeof(unsigned) * m), "counters")) != MLS_OK) return st;
  if ((st = up((void**)&B.chunk_beg, h_chunk_beg.data(), sizeof(int) * std::max(nchunk, 1))) != MLS_OK) return st;
  if ((st = up((void**)&B.slot_row, h_slot_row.data(), sizeof(int) * std::max(nbk, 1))) != MLS_OK) return st;
  B.m = m;
  B.nnz = nz;
  B.ny = ny;
  B.maxk = std::max(maxk, 1);
  B.nb = nbk;
  B.nent = (int64_t)nent;
  B.nchunk = nchunk;
  B.nrchunk = nrchunk;
  B.h_hrow = h_hrow;
  B.h_vrow = h_vrow;
  B.h_vh = h_vh;
  B.h_vphi = h_vphi;
  B.h_origins.assign(origins, origins + 3 * (size_t)m);
  const int r = 12 * m;
  const int vb = solve_bytes(ctx);
  // Y = H U and the Galerkin chunk partials are float64 in every precision
  if ((st = dalloc(ctx, &ctx->yval, (size_t)ny * 36 * sizeof(double))) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->gpart, (size_t)std::max(nchunk, 1) * 144 * sizeof(double))) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->Ac, (size_t)r * r * sizeof(double))) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->Acopy, (size_t)r * r * sizeof(double))) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->Linv, (size_t)r * r * vb)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->LinvT, (size_t)r * r * vb)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->Ainv, (size_t)r * r * vb)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->cvec, (size_t)r * vb)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->cvec2, (size_t)r * vb)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->chol_info, sizeof(int) * 4)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->oz_fwd, sizeof(__nv_bfloat16) * (size_t)r * kOzSlices * kOzPanel)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->oz_e, sizeof(int) * (size_t)r)) != MLS_OK) return st;
  if (!ctx->umma_err) {
    if ((st = dalloc(ctx, (void**)&ctx->umma_err, sizeof(int))) != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaMemset(ctx->umma_err, 0, sizeof(int)), "flag")) != MLS_OK) return st;
  }
  if ((st = dalloc(ctx, (void**)&ctx->chol_tinv, sizeof(double) * 32 * 32 * (size_t)((r + 31) / 32))) != MLS_OK)
    return st;
  ctx->has_basis = true;
  ctx->coarse_ready = false;
  ctx->galerkin_ready = false;
  return MLS_OK;
}

// ---- prolongation / restriction ---------------------------------------------------------
struct BasisView {
  int n, m;
  const void* __restrict__ vcoef;   // [nnz] (phi, phi a) vertex-major, solve precision
  const void* __restrict__ hcoef;   // [nnz] (phi, phi a) handle-major
  const int* __restrict__ rchunk_handle;
  const int* __restrict__ rchunk_beg;
  const int* __restrict__ rchunk_ptr;
  double* rpart;
  unsigned* rcount;
  const int* __restrict__ vrow;
  const int* __restrict__ vh;
  const double* __restrict__ vphi;
  const int* __restrict__ hrow;
  const int* __restrict__ hv;
  const double* __restrict__ hphi;
  const double* __restrict__ origins;
  const Vec4d* __restrict__ X;
  int nrchunk;
};

// sum_j phi_j(v) (I_3 (x) a_vj^T) q_j for one vertex: the handle indices and
// coefficients of four entries are loaded before their coarse vectors, so
// the dependent gathers of a row are issued together
template <typename VT>
__device__ __forceinline__ void prolong_row(const BasisView& B, const VT* __restrict__ q, int v, VT& o0, VT& o1,
                                            VT& o2) {
  const Vec4<VT>* coef = (const Vec4<VT>*)B.vcoef;
  const int k1 = B.vrow[v + 1];
  for (int k0 = B.vrow[v]; k0 < k1; k0 += 4) {
    int h[4];
    Vec4<VT> a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const bool ok = k0 + u < k1;
      h[u] = ok ? B.vh[k0 + u] : -1;
      a[u] = ok ? coef[k0 + u] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (h[u] < 0) continue;
      const Vec4<VT>* qj = (const Vec4<VT>*)(q + 12 * (int64_t)h[u]);
      const Vec4<VT> q0 = qj[0], q1 = qj[1], q2 = qj[2];
      o0 += a[u].x * q0.x + a[u].y * q0.y + a[u].z * q0.z + a[u].w * q0.w;
      o1 += a[u].x * q1.x + a[u].y * q1.y + a[u].z * q1.z + a[u].w * q1.w;
      o2 += a[u].x * q2.x + a[u].y * q2.y + a[u].z * q2.z + a[u].w * q2.w;
    }
  }
}

// half of the row: the vertex's handles at even (half = 0) or odd (half =
// 1) positions of its list, four at a time
template <typename VT>
__device__ __forceinline__ void prolong_row_half(const BasisView& B, const VT* __restrict__ q, int v, int half,
                                                 VT& o0, VT& o1, VT& o2) {
  const Vec4<VT>* coef = (const Vec4<VT>*)B.vcoef;
  const int k1 = B.vrow[v + 1];
  for (int k0 = B.vrow[v] + half; k0 < k1; k0 += 8) {
    int h[4];
    Vec4<VT> a[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 2 * u;
      const bool ok = k < k1;
      h[u] = ok ? B.vh[k] : -1;
      a[u] = ok ? coef[k] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (h[u] < 0) continue;
      const Vec4<VT>* qj = (const Vec4<VT>*)(q + 12 * (int64_t)h[u]);
      const Vec4<VT> q0 = qj[0], q1 = qj[1], q2 = qj[2];
      o0 += a[u].x * q0.x + a[u].y * q0.y + a[u].z * q0.z + a[u].w * q0.w;
      o1 += a[u].x * q1.x + a[u].y * q1.y + a[u].z * q1.z + a[u].w * q1.w;
      o2 += a[u].x * q2.x + a[u].y * q2.y + a[u].z * q2.z + a[u].w * q2.w;
    }
  }
}

// w_v = [acc ? w_v : 0] + sum_j phi_j(v) (I_3 (x) a_vj^T) q_j  (+ omega D^-1 s_v)
// (q may be null: then only the base and smoothing terms are applied; base
// and w may alias, each vertex's entry is read before it is written).  Two
// adjacent lanes per vertex split its handles and add their sums with one
// shuffle, so twice the threads keep the dependent gathers in flight.
// Launch with prolong_blocks(n).
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_prolong(BasisView B, const VT* __restrict__ q,
                                                    const Vec4<VT>* base,
                                                    const VT* __restrict__ dinv, const Vec4<VT>* __restrict__ s,
                                                    VT omega, Vec4<VT>* w,
                                                    const PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  if (S && S->done) return;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int v = (int)(gt >> 1), half = (int)(gt & 1);
  VT o0 = VT(0), o1 = VT(0), o2 = VT(0);
  if (q && v < B.n) prolong_row_half<VT>(B, q, v, half, o0, o1, o2);
  o0 += __shfl_xor_sync(0xffffffffu, o0, 1);
  o1 += __shfl_xor_sync(0xffffffffu, o1, 1);
  o2 += __shfl_xor_sync(0xffffffffu, o2, 1);
  if (v >= B.n || half) return;
  if (base) {
    const Vec4<VT> b = base[v];
    o0 += b.x; o1 += b.y; o2 += b.z;
  }
  if (s) {
    const Vec4<VT> sv = s[v];
    const VT* D = dinv + (int64_t)v * 9;
    o0 += omega * (D[0] * sv.x + D[1] * sv.y + D[2] * sv.z);
    o1 += omega * (D[3] * sv.x + D[4] * sv.y + D[5] * sv.z);
    o2 += omega * (D[6] * sv.x + D[7] * sv.y + D[8] * sv.z);
  }
  w[v] = Vec4<VT>{o0, o1, o2, VT(0)};
}

static inline int prolong_blocks(int n) { return nblk(2 * (int64_t)n); }

// z1 += U y in place, then r.z1 (the end of the additive cycle): inside the
// loop (first = 0, iteration it) into the sum that opens iteration it + 1,
// before it (first = 1) by a grid sum that sets rz_0
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_prolong_rz(BasisView B, const VT* __restrict__ q,
                                                       const Vec4<VT>* __restrict__ r, Vec4<VT>* z, int first,
                                                       int it, GridReduce gr, unsigned long long* __restrict__ fix,
                                                       PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  if (S->done) return;
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < B.n) {
    VT o0 = VT(0), o1 = VT(0), o2 = VT(0);
    prolong_row<VT>(B, q, v, o0, o1, o2);
    const Vec4<VT> zb = z[v], rv = r[v];
    const Vec4<VT> zo{zb.x + o0, zb.y + o1, zb.z + o2, VT(0)};
    z[v] = zo;
    acc[0] = (double)rv.x * zo.x + (double)rv.y * zo.y + (double)rv.z * zo.z;
  }
  if (!first) {
    __shared__ double sh[1][32];
    block_sum<1>(acc, sh);
    if (threadIdx.x == 0) fix_add(fix_slot(fix, FX_RZ, (it + 1) & 1), acc[0], fix_exponent(S->rzv[it & 1]));
    return;
  }
  if (grid_sum<1>(acc, gr, RS_PCG_RZ) && threadIdx.x == 0) {
    S->beta = 0.0;
    S->rz = acc[0];
    S->rzv[0] = acc[0];
    if (!(acc[0] > 0.0) || !isfinite(acc[0])) S->done = (S->rr <= S->tol2) ? 1 : 3;
  }
}

// z_j = sum_{v in supp j} phi_j(v) r_v (x) a_vj.  One warp per chunk of at
// most kRestrictChunk entries of one handle: each lane takes every 32nd
// entry (coalesced coefficients, eight independent gathers in flight), the
// warp sums its 12 values with shuffles, and the chunk sum goes to a
// per-chunk slot; the last chunk of a handle to finish adds the slots in
// chunk order (deterministic).  No block-wide barrier.
constexpr int kRestrictWarps = 8;
template <typename VT>
__global__ void __launch_bounds__(32 * kRestrictWarps) k_restrict(BasisView B, const Vec4<VT>* __restrict__ r,
                                                                  VT* __restrict__ z,
                                                                  const PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  if (S && S->done) return;
  const int lane = threadIdx.x & 31;
  const int ch = blockIdx.x * kRestrictWarps + (threadIdx.x >> 5);
  if (ch >= B.nrchunk) return;
  const int j = B.rchunk_handle[ch];
  const int p0 = B.rchunk_beg[ch];
  const int p1 = min(p0 + kRestrictChunk, B.hrow[j + 1]);
  constexpr int U = kRestrictChunk / 32;
  int hv[U];
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int p = p0 + lane + 32 * u;
    hv[u] = p < p1 ? B.hv[p] : -1;
  }
  VT acc[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) acc[q] = VT(0);
#pragma unroll
  for (int u = 0; u < U; ++u) {
    if (hv[u] < 0) continue;
    const Vec4<VT> a = ((const Vec4<VT>*)B.hcoef)[p0 + lane + 32 * u];
    const Vec4<VT> rv = r[hv[u]];
    const VT rc[3] = {rv.x, rv.y, rv.z};
    const VT av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int l = 0; l < 4; ++l) acc[4 * c + l] += rc[c] * av[l];
  }
#pragma unroll
  for (int q = 0; q < 12; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
  // lane q < 12 stores component q (the values are identical in every lane)
  VT mine = acc[0];
#pragma unroll
  for (int q = 1; q < 12; ++q)
    if (lane == q) mine = acc[q];
  if (lane < 12) B.rpart[12 * (int64_t)ch + lane] = (double)mine;
  __syncwarp();
  unsigned last = 0;
  if (lane == 0) {
    __threadfence();
    const unsigned nch = (unsigned)(B.rchunk_ptr[j + 1] - B.rchunk_ptr[j]);
    last = atomicAdd(B.rcount + j, 1u) == nch - 1;
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return;
  __threadfence();
  if (lane < 12) {
    const double t = ordered_sum_ldcg(B.rpart + lane, 12, B.rchunk_ptr[j], B.rchunk_ptr[j + 1]);
    z[12 * (int64_t)j + lane] = (VT)t;
  }
  if (lane == 0) B.rcount[j] = 0;
}

static inline int restrict_blocks(int nrchunk) { return (nrchunk + kRestrictWarps - 1) / kRestrictWarps; }

// ---- Galerkin: Y = H U ----------------------------------------------------------------
struct GalerkinView {
  int n;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ col;
  const int* __restrict__ row_len;
  const int* __restrict__ yrow;
  const int* __restrict__ yh;
  const int16_t* __restrict__ yslot;
  int maxk;
};

// one thread per (v, local handle q of K_v); Y stored [ny][36]
template <typename VT, typename MT>
__global__ void __launch_bounds__(kBlock) k_galerkin_y(BasisView B, GalerkinView G, const MT* __restrict__ val,
                                                       const int* __restrict__ ypair_row, int64_t ny,
                                                       VT* __restrict__ Y) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ny) return;
  const int v = ypair_row[idx];
  const int q = (int)(idx - G.yrow[v]);
  const int j = G.yh[idx];
  const double ox = B.origins[3 * j], oy = B.origins[3 * j + 1], oz = B.origins[3 * j + 2];
  VT acc[36];
#pragma unroll
  for (int k = 0; k < 36; ++k) acc[k] = VT(0);
  const int slice = v >> 5, lane = v & 31;
  const int g0 = G.slice_ptr[slice];
  const int len = G.row_len[v];
  for (int k = 0; k < len; ++k) {
    const int64_t slot = ((int64_t)g0 + k) * 32 + lane;
    const int w = G.col[slot];
    const int kb = B.vrow[w], ke = B.vrow[w + 1];
    for (int e = kb; e < ke; ++e) {
      if (G.yslot[slot * G.maxk + (e - kb)] != q) continue;
      const Vec4d Xw = B.X[w];
      const VT ph = (VT)B.vphi[e];
      const VT a[4] = {ph, ph * (VT)(Xw.x - ox), ph * (VT)(Xw.y - oy), ph * (VT)(Xw.z - oz)};
      const MT* hv = val + ((int64_t)g0 + k) * 288 + lane;
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const VT h = load_as<VT>(hv[(3 * c + d) * 32]);
#pragma unroll
          for (int l = 0; l < 4; ++l) acc[(3 * c + d) * 4 + l] += h * a[l];
        }
    }
  }
#pragma unroll
  for (int k = 0; k < 36; ++k) Y[idx * 36 + k] = acc[k];
}

// The same Y = H U in float64, one warp per vertex row v: the warp walks the
// row's blocks H_vw in slot order; for each block, lanes 0..26 take one of
// the nine values H_vw[c][d] for one of three basis entries (j, phi_j(w)) of
// w at a time and add H_vw[c][d] phi_j(w) a_l(w) (l = 0..3) to the row's
// accumulator for handle j, which lives in shared memory (K_v x 36 doubles
// per warp).  The entries of one block belong to different handles, so no
// two lanes update the same word, and the blocks are added in slot order:
// the sums are deterministic.  Every lane of the warp does the same loop
// trip count, so the float64 work is not serialised by divergence.
constexpr int kGalYWarps = 4;
template <typename MT>
__global__ void __launch_bounds__(32 * kGalYWarps) k_galerkin_y64(BasisView B, GalerkinView G,
                                                                 const MT* __restrict__ val, int maxkv,
                                                                 double* __restrict__ Y) {
  extern __shared__ double s_yacc[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int v = blockIdx.x * kGalYWarps + warp;
  if (v >= G.n) return;
  double* acc = s_yacc + (size_t)warp * maxkv * 36;
  const int y0 = G.yrow[v], kv = G.yrow[v + 1] - y0;
  for (int t = lane; t < kv * 36; t += 32) acc[t] = 0.0;
  __syncwarp();
  const int cd = lane % 9, eo = lane / 9;  // eo = 3: lanes 27..31 only help with the final copy
  const int slice = v >> 5, sl = v & 31;
  const int g0 = G.slice_ptr[slice];
  const int len = G.row_len[v];
  for (int k = 0; k < len; ++k) {
    const int64_t slot = ((int64_t)g0 + k) * 32 + sl;
    const int w = G.col[slot];
    const int kb = B.vrow[w], ke = B.vrow[w + 1];
    if (eo < 3) {
      const double h = load_as<double>(val[((int64_t)g0 + k) * 288 + cd * 32 + sl]);
      const Vec4d Xw = B.X[w];
      for (int e = kb + eo; e < ke; e += 3) {
        const int q = G.yslot[slot * G.maxk + (e - kb)];
        const int j = B.vh[e];
        const double ph = B.vphi[e];
        double* a = acc + q * 36 + cd * 4;
        a[0] += h * ph;
        a[1] += h * (ph * (Xw.x - B.origins[3 * j]));
        a[2] += h * (ph * (Xw.y - B.origins[3 * j + 1]));
        a[3] += h * (ph * (Xw.z - B.origins[3 * j + 2]));
      }
    }
    __syncwarp();
  }
  for (int t = lane; t < kv * 36; t += 32) Y[(int64_t)y0 * 36 + t] = acc[t];
}

// A_ij (12x12) = sum over entries (v, y) of phi_i(v) a_vi (x) Y_y.  Pass 1:
// one 144-thread team per chunk of at most kGalerkinChunk entries of one
// coarse block (two teams per CTA), each thread owning one of the 144
// outputs; the chunk's entry metadata is staged in shared memory.
template <typename VT>
__global__ void __launch_bounds__(288) k_galerkin_chunk(BasisView B, const int* __restrict__ chunk_beg,
                                                        const int* __restrict__ chunk_ptr,
                                                        const int* __restrict__ slot_row, int nbk,
                                                        const int* __restrict__ ent_ptr,
                                                        const int* __restrict__ ent_y,
                                                        const int* __restrict__ ent_v,
                                                        const double* __restrict__ ent_phi, int nchunk,
                                                        const VT* __restrict__ Y, VT* __restrict__ part) {
  __shared__ int s_y[2][kGalerkinChunk];
  __shared__ VT s_coef[2][kGalerkinChunk][4];
  const int team = threadIdx.x / 144, tt = threadIdx.x % 144;
  const int chunk = blockIdx.x * 2 + team;
  const bool active = chunk < nchunk;
  int beg = 0, end = 0, i = 0;
  if (active) {
    // slot of this chunk: last slot whose first chunk is <= chunk (binary search)
    int lo = 0, hi = nbk - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (chunk_ptr[mid] <= chunk) lo = mid; else hi = mid - 1;
    }
    beg = chunk_beg[chunk];
    end = min(beg + kGalerkinChunk, ent_ptr[lo + 1]);
    i = slot_row[lo];
  }
  if (active) {
    const double ox = B.origins[3 * i], oy = B.origins[3 * i + 1], oz = B.origins[3 * i + 2];
    for (int p = beg + tt; p < end; p += 144) {
      const int q = p - beg;
      const int v = ent_v[p];
      const Vec4d X = B.X[v];
      const double ph = ent_phi[p];
      s_y[team][q] = ent_y[p];
      s_coef[team][q][0] = (VT)ph;
      s_coef[team][q][1] = (VT)(ph * (X.x - ox));
      s_coef[team][q][2] = (VT)(ph * (X.y - oy));
      s_coef[team][q][3] = (VT)(ph * (X.z - oz));
    }
  }
  __syncthreads();
  if (!active) return;
  const int row = tt / 12, colq = tt % 12;  // row = 4 c + l', col = 4 d + l
  const int c = row >> 2, lp = row & 3, d = colq >> 2, l = colq & 3;
  const int yk = (3 * c + d) * 4 + l;
  VT acc = VT(0);
  const int cnt = end - beg;
#pragma unroll 4
  for (int q = 0; q < cnt; ++q) acc += s_coef[team][q][lp] * Y[(int64_t)s_y[team][q] * 36 + yk];
  part[(int64_t)chunk * 144 + tt] = acc;
}

// Pass 2: each coarse block sums its chunks in order and writes A (float64)
template <typename VT>
__global__ void __launch_bounds__(144) k_galerkin_reduce(const int* __restrict__ chunk_ptr,
                                                         const int* __restrict__ slot_row,
                                                         const int* __restrict__ hn, const VT* __restrict__ part,
                                                         int r, double* __restrict__ A) {
  const int sl = blockIdx.x;
  const int tt = threadIdx.x;
  double acc = 0.0;
  for (int ch = chunk_ptr[sl]; ch < chunk_ptr[sl + 1]; ++ch) acc += (double)part[(int64_t)ch * 144 + tt];
  const int i = slot_row[sl], j = hn[sl];
  A[(int64_t)(12 * i + tt / 12) * r + 12 * j + tt % 12] = acc;
}

// ---- dense Cholesky (float64), blocked right-looking ---------------------------------------
constexpr int NB = 32;

// 1/sqrt(d) for a positive float64 d: a float seed (rsqrtf) refined by two
// Newton steps on f(y) = 1/y^2 - d, y <- y + y (1 - d y^2) / 2.  Each step
// squares the relative error: the seed's ~2^-22 becomes ~2^-44 and then
// falls below float64 rounding.  Outside the float range of the seed the
// library's own 1/sqrt is taken.
__device__ __forceinline__ double rsqrt_refined(double d) {
  if (!(d > 1e-30 && d < 1e30)) return 1.0 / sqrt(d);
  double y = (double)rsqrtf((float)d);
  const double hd = 0.5 * d;
#pragma unroll
  for (int it = 0; it < 2; ++it) y = fma(y, fma(-hd * y, y, 0.5), y);
  return y;
}

// pivot p of a diagonal tile: d = a_pp after the p earlier elimination
// steps; records the first non-positive pivot in info and continues with 1
__device__ __forceinline__ void tile_pivot(double d, int p, int base, int* __restrict__ info,
                                           double* __restrict__ rd, double* __restrict__ rd2) {
  if (!(d > 0.0)) {
    if (*info == 0) *info = base + p + 1;
    d = 1.0;
  }
  const double y = rsqrt_refined(d);
  rd[p] = y;       // 1/sqrt(a_pp)
  rd2[p] = y * y;  // 1/a_pp
}

// Factor the diagonal tile (k, k) in place (lower factor; upper part set to
// 0) and write the inverse of that factor to tinv[k] (32 x 32, row-major).
// Right-looking elimination on the unscaled tile: step p subtracts
// m_ip * (row p) from every row i > p of the trailing part, m_ip = a_ip / a_pp,
// and applies the same row operation to G (initially I).  Afterwards
// A = Lt D Lt^T with unit lower Lt, G = Lt^{-1} and D the pivots, so
// L = Lt D^{1/2} (L_ij = a_ij / sqrt(a_jj), the column scaled once at the
// end) and L^{-1} = D^{-1/2} G.  The G update takes the lanes left of column
// p that the trailing update leaves idle.  Thread (ty, tx) owns element
// (ty, tx) of both; the thread that produces a_{p+1,p+1} computes the next
// pivot at once, so each column costs one barrier.  One CTA of 32x32 threads.
__global__ void k_potrf_tile(double* __restrict__ A, int r, int k, int* __restrict__ info,
                             double* __restrict__ tinv) {
  __shared__ double T[NB][NB + 1];
  __shared__ double G[NB][NB + 1];
  __shared__ double rd[NB], rd2[NB];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int base = k * NB;
  const int nr = min(NB, r - base);
  T[ty][tx] = (ty < nr && tx < nr) ? A[(int64_t)(base + ty) * r + base + tx] : (ty == tx ? 1.0 : 0.0);
  G[ty][tx] = (ty == tx) ? 1.0 : 0.0;
  if (ty == 0) { rd[tx] = 1.0; rd2[tx] = 1.0; }  // rows past the matrix edge
  __syncthreads();
  if (tx == 0 && ty == 0) tile_pivot(T[0][0], 0, base, info, rd, rd2);
  __syncthreads();
  for (int p = 0; p < nr; ++p) {
    if (ty > p) {
      const double m = T[ty][p] * rd2[p];
      if (tx > p) {
        if (tx <= ty) {
          const double v = fma(-m, T[tx][p], T[ty][tx]);
          T[ty][tx] = v;
          if (tx == p + 1 && ty == p + 1 && p + 1 < nr) tile_pivot(v, p + 1, base, info, rd, rd2);
        }
      } else if (tx < p) {
        G[ty][tx] = fma(-m, G[p][tx], G[ty][tx]);
      } else {
        G[ty][p] = -m;
      }
    }
    __syncthreads();
  }
  if (ty < nr && tx < nr) A[(int64_t)(base + ty) * r + base + tx] = (tx <= ty) ? T[ty][tx] * rd[tx] : 0.0;
  tinv[(int64_t)k * NB * NB + ty * NB + tx] = (tx < ty) ? G[ty][tx] * rd[ty] : (tx == ty ? rd[ty] : 0.0);
}

// L_ik = A_ik L_kk^{-T} = A_ik (tinv)^T for tiles i > k; one CTA (32x32) per tile
__global__ void k_trsm_tiles(double* __restrict__ A, int r, int k, const double* __restrict__ tinv) {
  __shared__ double Li[NB][NB + 1];
  __shared__ double X[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i = k + 1 + blockIdx.x;
  const int bk = k * NB, bi = i * NB;
  const int nk = min(NB, r - bk), ni = min(NB, r - bi);
  Li[ty][tx] = tinv[(int64_t)k * NB * NB + ty * NB + tx];
  X[ty][tx] = (ty < ni && tx < nk) ? A[(int64_t)(bi + ty) * r + bk + tx] : 0.0;
  __syncthreads();
  double s = 0.0;
#pragma unroll 8
  for (int q = 0; q <= tx; ++q) s += X[ty][q] * Li[tx][q];
  if (ty < ni && tx < nk) A[(int64_t)(bi + ty) * r + bk + tx] = s;
}

// A_ij -= L_ik L_jk^T for k < j <= i (lower triangle of the trailing matrix);
// one CTA (32x8 threads, 4 outputs each) per tile pair
__global__ void k_syrk_tiles(double* __restrict__ A, int r, int k, int ntiles) {
  // map blockIdx.x to (i, j) with k < j <= i < ntiles
  const int m = ntiles - k - 1;
  int idx = blockIdx.x;
  int jj = 0;
  while (idx >= m - jj) { idx -= m - jj; ++jj; }
  const int j = k + 1 + jj;
  const int i = j + idx;
  __shared__ double Li[NB][NB + 1];
  __shared__ double Lj[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  const int bk = k * NB, bi = i * NB, bj = j * NB;
  const int nk = min(NB, r - bk), ni = min(NB, r - bi), nj = min(NB, r - bj);
  for (int rr = ty; rr < NB; rr += 8) {
    Li[rr][tx] = (rr < ni && tx < nk) ? A[(int64_t)(bi + rr) * r + bk + tx] : 0.0;
    Lj[rr][tx] = (rr < nj && tx < nk) ? A[(int64_t)(bj + rr) * r + bk + tx] : 0.0;
  }
  __syncthreads();
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < NB; ++q) {
    const double b = Lj[tx][q];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += Li[ty + 8 * u][q] * b;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = ty + 8 * u;
    if (rr < ni && tx < nj) A[(int64_t)(bi + rr) * r + bj + tx] -= acc[u];
  }
}

// ---- float64 trailing updates on the tensor cores ------------------------------------
// The rank-128 update A22 -= L21 L21^T of the blocked Cholesky is computed
// as an error-free sum of bf16 products (the splitting scheme of Ozaki,
// Ogita, Oishi and Rump, 2012): each row i of L21 is scaled by 2^-e_i (e_i
// the exponent of its largest entry, so the row lies in (-1, 1)) and cut
// into kOzSlices slices of kOzBits bits, a_p = trunc(2^beta r_{p-1}),
// r_p = 2^beta r_{p-1} - a_p (exact in float64).  Every slice entry is an
// integer of magnitude < 2^7, exact in bf16, and a product of two slices
// summed over at most 1024 terms stays below 2^24, exact in the float32
// accumulator.  So S_d = sum_{p+q=d} a_p a_q^T, each a sum of tensor-core
// products of slice pairs, is exact, and
//   (L21 L21^T)_ij = 2^(e_i + e_j) sum_d 2^(-beta d) S_d,ij
// up to the dropped terms p + q > kOzSlices + 1, below 2^-56 relative to the
// row scales.  The S_d are formed together (k_ozaki_syrk, umma.cu), scaled
// exactly by powers of two, summed and subtracted from A22 in float64.
// slices of the rows of an FP64 block [rows][K] (pitch lda), slice p at
// columns p K of fwd (row pitch opitch); the row exponents to e
__global__ void k_ozaki_split(int rows, int K, const double* __restrict__ A, int lda, int opitch,
                              __nv_bfloat16* __restrict__ fwd, int* __restrict__ e) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= rows) return;
  const double* a = A + (int64_t)i * lda;
  double mx = 0.0;
  for (int k = lane; k < K; k += 32) mx = fmax(mx, fabs(a[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  int ex = 0;
  if (mx > 0.0) frexp(mx, &ex);  // mx = f 2^ex, f in [0.5, 1): every |a_k| < 2^ex
  if (lane == 0) e[i] = ex;
  __nv_bfloat16* f = fwd + (int64_t)i * opitch;
  for (int k = lane; k < K; k += 32) {
    double r = ldexp(a[k], -ex);
#pragma unroll
    for (int p = 0; p < kOzSlices; ++p) {
      r = ldexp(r, kOzBits);
      const double t = trunc(r);
      r -= t;
      const __nv_bfloat16 v = __double2bfloat16(t);
      f[p * K + k] = v;
    }
  }
}

// A[r1:, r1:] -= L21 L21^T (lower triangle), L21 = A[r1:, c0:c0+w], w <= 128
static mls_status ozaki_trailing_update(mls_ctx* ctx, double* A, int r, int c0, int w, int r1) {
  const int n = r - r1;
  if (n <= 0) return MLS_OK;
  const int opitch = kOzSlices * kOzPanel;
  { ++ctx->launches; k_ozaki_split<<<(n + 7) / 8, 256, 0, ctx->stream>>>(n, w, A + (int64_t)r1 * r + c0, r, opitch,
                                                                        ctx->oz_fwd, ctx->oz_e); }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "k_ozaki_split");
  if (st != MLS_OK) return st;
  if (w != kOzPanel) return fail(ctx, MLS_EINVAL, "tensor-core trailing update: panel width");
  ++ctx->launches;
  st = ozaki_syrk(ctx->stream, n, ctx->oz_fwd, opitch, ctx->oz_e, A + (int64_t)r1 * r + r1, r, ctx->umma_err);
  if (st != MLS_OK) return fail(ctx, st, "tensor-core trailing update");
  return MLS_OK;
}

// W = L^{-1} by a right-looking blocked solve of L W = I over tile rows:
// step i solves the tile row in place, W_ic = L_ii^{-1} B_ic for c <= i, with
// the diagonal tile's inverse from the factorisation (k_trinv_solve), then
// updates the rows below, B_qc -= L_qi W_ic for q > i, c <= i
// (k_trinv_update).  W starts as the identity; its upper part stays 0.
template <typename VT>
__global__ void k_eye(VT* __restrict__ W, int r) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < r) W[k * r + k] = VT(1);
}

// W_ic = tinv[i] B_ic for one column tile c <= i; one CTA of 32x32 threads
template <typename VT>
__global__ void k_trinv_solve(const double* __restrict__ tinv, int r, int i, VT* __restrict__ W) {
  __shared__ VT Ti[NB][NB + 1];
  __shared__ VT X[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int c = blockIdx.x;  // column tile, c <= i
  const int bi = i * NB, bc = c * NB;
  const int ni = min(NB, r - bi), nc = min(NB, r - bc);
  Ti[ty][tx] = (VT)tinv[(int64_t)i * NB * NB + ty * NB + tx];
  X[ty][tx] = (ty < ni && tx < nc) ? W[(int64_t)(bi + ty) * r + bc + tx] : VT(0);
  __syncthreads();
  VT v = VT(0);
#pragma unroll 8
  for (int q = 0; q <= ty; ++q) v += Ti[ty][q] * X[q][tx];
  if (ty < ni && tx < nc) W[(int64_t)(bi + ty) * r + bc + tx] = v;
}

// B_qc -= L_qi W_ic for q in (i, nt), c in [0, i]; one CTA (32x8 threads,
// 4 outputs each) per (q, c) tile
template <typename VT>
__global__ void k_trinv_update(const double* __restrict__ L, int r, int i, int nt, VT* __restrict__ W) {
  const int q = i + 1 + blockIdx.x / (i + 1);
  const int c = blockIdx.x % (i + 1);
  __shared__ VT Lq[NB][NB + 1];
  __shared__ VT Wi[NB][NB + 1];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int bq = q * NB, bi = i * NB, bc = c * NB;
  const int nq = min(NB, r - bq), ni = min(NB, r - bi), nc = min(NB, r - bc);
  for (int rr = ty; rr < NB; rr += 8) {
    Lq[rr][tx] = (rr < nq && tx < ni) ? (VT)L[(int64_t)(bq + rr) * r + bi + tx] : VT(0);
    Wi[rr][tx] = (rr < ni && tx < nc) ? W[(int64_t)(bi + rr) * r + bc + tx] : VT(0);
  }
  __syncthreads();
  VT acc[4] = {VT(0), VT(0), VT(0), VT(0)};
#pragma unroll 8
  for (int k = 0; k < NB; ++k) {
    const VT b = Wi[k][tx];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] += Lq[ty + 8 * u][k] * b;
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int rr = ty + 8 * u;
    if (rr < nq && tx < nc) W[(int64_t)(bq + rr) * r + bc + tx] -= acc[u];
  }
}

// WT = W^T, 32x32 tiles through shared memory
template <typename VT>
__global__ void k_transpose(const VT* __restrict__ W, int r, VT* __restrict__ WT) {
  __shared__ VT T[NB][NB + 1];
  const int bx = blockIdx.x * NB, by = blockIdx.y * NB;
  for (int k = threadIdx.y; k < NB; k += blockDim.y) {
    const int rr = by + k, cc = bx + threadIdx.x;
    T[k][threadIdx.x] = (rr < r && cc < r) ? W[(int64_t)rr * r + cc] : VT(0);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < NB; k += blockDim.y) {
    const int rr = bx + k, cc = by + threadIdx.x;
    if (rr < r && cc < r) WT[(int64_t)rr * r + cc] = T[threadIdx.x][k];
  }
}

// C = W^T W for lower-triangular W (r x r): the inverse of the coarse
// operator, A^{-1} = L^{-T} L^{-1}.  64 x 64 output tiles (I, J), J <= I, each
// also written mirrored; 256 threads, 4 x 4 outputs each; rows k of W below
// the tile's first row I*64 are zero in column block I and skipped.
constexpr int kGramTile = 64;
template <typename VT>
__global__ void __launch_bounds__(256) k_gram_lower(const VT* __restrict__ W, int r, VT* __restrict__ C) {
  const int T = (r + kGramTile - 1) / kGramTile;
  int idx = blockIdx.x, I = 0;
  while (idx > I) { idx -= I + 1; ++I; }
  const int J = idx;  // 0 <= J <= I < T
  (void)T;
  __shared__ VT As[16][kGramTile];
  __shared__ VT Bs[16][kGramTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  VT acc[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = VT(0);
  const int i0 = I * kGramTile, j0 = J * kGramTile;
  for (int k0 = i0; k0 < r; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * kGramTile; e += 256) {
      const int kk = e / kGramTile, c = e % kGramTile;
      const int k = k0 + kk;
      As[kk][c] = (k < r && i0 + c < r) ? W[(int64_t)k * r + i0 + c] : VT(0);
      Bs[kk][c] = (k < r && j0 + c < r) ? W[(int64_t)k * r + j0 + c] : VT(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 16; ++kk) {
      VT a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = As[kk][ty * 4 + u]; b[u] = Bs[kk][tx * 4 + u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] += a[u] * b[v];
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = i0 + ty * 4 + u, j = j0 + tx * 4 + v;
      if (i < r && j < r) {
        C[(int64_t)i * r + j] = acc[u][v];
        C[(int64_t)j * r + i] = acc[u][v];
      }
    }
}

// y = W x restricted to the lower (lower = 1: columns <= row) or upper
// (lower = 0: columns >= row) triangle, widened to 16-byte boundaries (W is
// zero outside its triangle); lower = 2: the whole row (dense W).  kTriWarps warps share a row (lane-strided
// 16-byte loads, so each warp has few loads to wait for) and combine their
// sums through shared memory; a 256-thread block covers 8 / kTriWarps rows.
constexpr int kTriWarps = 4;
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_trigemv(const VT* __restrict__ W, int r, int lower,
                                                    const VT* __restrict__ x, VT* __restrict__ y,
                                                    const PcgScalars* __restrict__ S) {
  chain_wait();
  chain_release();
  if (S && S->done) return;
  constexpr int EV = 16 / sizeof(VT);
  constexpr int RPB = (kBlock / 32) / kTriWarps;
  __shared__ VT part[kBlock / 32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * RPB + warp / kTriWarps;
  const int sub = warp % kTriWarps;
  VT acc = VT(0);
  if (row < r) {
    const int v0 = lower ? 0 : row / EV;
    const int v1 = lower == 1 ? (row + EV) / EV : r / EV;
    using V16 = typename std::conditional<sizeof(VT) == 4, float4, double2>::type;
    const V16* Wr = reinterpret_cast<const V16*>(W + (int64_t)row * r);
    const V16* xv = reinterpret_cast<const V16*>(x);
#pragma unroll 4
    for (int c = v0 + sub * 32 + lane; c < v1; c += 32 * kTriWarps) {
      const V16 w = Wr[c];
      const V16 b = xv[c];
      if constexpr (sizeof(VT) == 4) {
        acc += w.x * b.x + w.y * b.y + w.z * b.z + w.w * b.w;
      } else {
        acc += w.x * b.x + w.y * b.y;
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (sub == 0 && lane == 0 && row < r) {
    VT t = VT(0);
#pragma unroll
    for (int k = 0; k < kTriWarps; ++k) t += part[warp + k];
    y[row] = t;
  }
}

static inline int trigemv_blocks(int r) {
  constexpr int RPB = (kBlock / 32) / kTriWarps;
  return (r + RPB - 1) / RPB;
}

__global__ void k_ypair_rows(int n, const int* __restrict__ yrow, int* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  for (int k = yrow[v]; k < yrow[v + 1]; ++k) out[k] = v;
}

// ---- host drivers --------------------------------------------------------------------------
static BasisView basis_view(mls_ctx* ctx) {
  const Basis& B = ctx->basis;
  return BasisView{ctx->n, B.m, B.vcoef, B.hcoef, B.rchunk_handle, B.rchunk_beg, B.rchunk_ptr, B.rpart, B.rcount,
                   B.vrow, B.vh, B.vphi, B.hrow, B.hv, B.hphi, B.origins, ctx->X, B.nrchunk};
}

mls_status launch_prolong(mls_ctx* ctx, const void* q, void* w, bool accumulate) {
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_prolong<double><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(basis_view(ctx), (const double*)q,
        accumulate ? (const Vec4d*)w : nullptr, nullptr, nullptr, 0.0, (Vec4d*)w, nullptr); }
  else
    { ++ctx->launches; k_prolong<float><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(basis_view(ctx), (const float*)q,
        accumulate ? (const Vec4f*)w : nullptr, nullptr, nullptr, 0.0f, (Vec4f*)w, nullptr); }
  return cuda_check(ctx, cudaGetLastError(), "k_prolong");
}

mls_status launch_restrict(mls_ctx* ctx, const void* r, void* q) {
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_restrict<double><<<restrict_blocks(ctx->basis.nrchunk), 32 * kRestrictWarps, 0, ctx->stream>>>(basis_view(ctx), (const Vec4d*)r, (double*)q, nullptr); }
  else
    { ++ctx->launches; k_restrict<float><<<restrict_blocks(ctx->basis.nrchunk), 32 * kRestrictWarps, 0, ctx->stream>>>(basis_view(ctx), (const Vec4f*)r, (float*)q, nullptr); }
  return cuda_check(ctx, cudaGetLastError(), "k_restrict");
}

// A_c = U^T H U accumulated in float64 from H's stored values (float64,
// float32 or bfloat16): the coarse operator's smallest eigenvalues are
// differences of large terms (near-rigid motions of stiff regions, whose
// elastic parts cancel down to the mass), and float32 sums of those terms
// can leave U^T H U indefinite when the stiffness contrast is large.
template <typename VT, typename MT>
static mls_status galerkin_t(mls_ctx* ctx) {
  Basis& B = ctx->basis;
  const int r = 12 * B.m;
  // Y = H U over H's element pattern; the cross-body contact blocks in the
  // spare slots past it are added separately (contact_galerkin)
  const int* rl0 = ctx->cs.row_len0 ? ctx->cs.row_len0 : ctx->row_len;
  GalerkinView G{ctx->n, ctx->slice_ptr, ctx->col, rl0, B.yrow, B.yh, B.yslot, B.maxk};
  if (!B.ypair_row) {
    mls_status st = dalloc(ctx, (void**)&B.ypair_row, sizeof(int) * std::max<int64_t>(B.ny, 1));
    if (st != MLS_OK) return st;
    { ++ctx->launches; k_ypair_rows<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, B.yrow, B.ypair_row); }
  }
  // with a cubature the coarse operator is built from the cubature H (Sec. 3.8)
  const MT* hv = (const MT*)(ctx->cub_scale ? ctx->hval_cub : ctx->hval);
  // the warp-per-row kernel while its accumulators fit in shared memory
  const size_t ysmem = (size_t)kGalYWarps * std::max(B.maxkv, 1) * 36 * sizeof(double);
  if (std::is_same<VT, double>::value && ysmem <= 200 * 1024) {
    if (ysmem > 48 * 1024) {
      mls_status st0 = cuda_check(ctx, cudaFuncSetAttribute(k_galerkin_y64<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                            (int)ysmem), "galerkin smem");
      if (st0 != MLS_OK) return st0;
    }
    { ++ctx->launches; k_galerkin_y64<MT><<<(ctx->n + kGalYWarps - 1) / kGalYWarps, 32 * kGalYWarps, ysmem, ctx->stream>>>(
        basis_view(ctx), G, hv, std::max(B.maxkv, 1), (double*)ctx->yval); }
  } else {
    { ++ctx->launches; k_galerkin_y<VT, MT><<<nblk(B.ny), kBlock, 0, ctx->stream>>>(basis_view(ctx), G, hv,
                                                                 B.ypair_row, B.ny, (VT*)ctx->yval); }
  }
  mls_status st = cuda_check(ctx, cudaMemsetAsync(ctx->Ac, 0, sizeof(double) * r * r, ctx->stream), "Ac clear");
  if (st != MLS_OK) return st;
  if (B.nchunk > 0) {
    { ++ctx->launches; k_galerkin_chunk<VT><<<(B.nchunk + 1) / 2, 288, 0, ctx->stream>>>(
        basis_view(ctx), B.chunk_beg, B.chunk_ptr, B.slot_row, B.nb, B.ent_ptr, B.ent_y, B.ent_v, B.ent_phi,
        B.nchunk, (const VT*)ctx->yval, (VT*)ctx->gpart); }
    { ++ctx->launches; k_galerkin_reduce<VT><<<B.nb, 144, 0, ctx->stream>>>(B.chunk_ptr, B.slot_row, B.hn,
                                                                            (const VT*)ctx->gpart, r, ctx->Ac); }
  }
  st = cuda_check(ctx, cudaGetLastError(), "galerkin");
  if (st != MLS_OK) return st;
  return contact_galerkin(ctx, hv);
}

// Factor the dense SPD float64 matrix A (r x r, row-major, overwritten by
// its Cholesky factor in the lower triangle) and form W = L^{-1} and W^T in
// solve precision.  Acopy (nullable) receives A before factorisation.
template <typename VT>
static mls_status factor_dense_t(mls_ctx* ctx, double* A, int r, double* Acopy, void* W, void* WT) {
  const int nt = (r + NB - 1) / NB;
  mls_status st;
  if (Acopy) {
    st = cuda_check(ctx, cudaMemcpyAsync(Acopy, A, sizeof(double) * r * r, cudaMemcpyDeviceToDevice, ctx->stream),
                    "A copy");
    if (st != MLS_OK) return st;
  }
  st = cuda_check(ctx, cudaMemsetAsync(ctx->chol_info, 0, sizeof(int), ctx->stream), "info clear");
  if (st != MLS_OK) return st;
  // Above kOzMinTiles tiles the factorisation goes by 128-wide panels: the
  // tile steps inside a panel update only the panel's own columns, and the
  // rest of the trailing matrix takes the panel's rank-128 update on the
  // tensor cores at the panel's end (the same sum of updates, delayed).
  constexpr int kOzMinTiles = 8;
  const int tpp = kOzPanel / NB;  // tiles per panel
  const bool oz = nt > kOzMinTiles && ctx->oz_fwd;
  for (int k = 0; k < nt; ++k) {
    { ++ctx->launches; k_potrf_tile<<<1, dim3(NB, NB), 0, ctx->stream>>>(A, r, k, ctx->chol_info, ctx->chol_tinv); }
    if (k + 1 < nt) {
      { ++ctx->launches; k_trsm_tiles<<<nt - k - 1, dim3(NB, NB), 0, ctx->stream>>>(A, r, k, ctx->chol_tinv); }
      // tile pairs (i, j), k < j < jmax, j <= i < nt
      const int jmax = oz ? std::min(nt, (k / tpp + 1) * tpp) : nt;
      int pairs = 0;
      for (int j = k + 1; j < jmax; ++j) pairs += nt - j;
      if (pairs > 0) { ++ctx->launches; k_syrk_tiles<<<pairs, dim3(32, 8), 0, ctx->stream>>>(A, r, k, nt); }
      if (oz && k + 1 == jmax && jmax < nt) {
        const int c0 = (jmax - tpp) * NB;
        if ((st = ozaki_trailing_update(ctx, A, r, c0, kOzPanel, jmax * NB)) != MLS_OK) return st;
      }
    }
  }
  st = cuda_check(ctx, cudaGetLastError(), "cholesky");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemsetAsync(W, 0, (size_t)r * r * sizeof(VT), ctx->stream), "W clear");
  if (st != MLS_OK) return st;
  { ++ctx->launches; k_eye<VT><<<(r + 255) / 256, 256, 0, ctx->stream>>>((VT*)W, r); }
  for (int i = 0; i < nt; ++i) {
    { ++ctx->launches; k_trinv_solve<VT><<<i + 1, dim3(NB, NB), 0, ctx->stream>>>(ctx->chol_tinv, r, i, (VT*)W); }
    if (i + 1 < nt) {
      { ++ctx->launches; k_trinv_update<VT><<<(nt - i - 1) * (i + 1), dim3(32, 8), 0, ctx->stream>>>(A, r, i, nt, (VT*)W); }
    }
  }
  { ++ctx->launches; k_transpose<VT><<<dim3(nt, nt), dim3(32, 8), 0, ctx->stream>>>((const VT*)W, r, (VT*)WT); }
  st = cuda_check(ctx, cudaGetLastError(), "triangular inverse");
  if (st != MLS_OK) return st;
  int info = 0;
  st = cuda_check(ctx, cudaMemcpyAsync(&ctx->dscal_host[12], ctx->chol_info, sizeof(int),
                                       cudaMemcpyDeviceToHost, ctx->stream), "info readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "cholesky sync");
  if (st != MLS_OK) return st;
  memcpy(&info, &ctx->dscal_host[12], sizeof(int));
  if (oz) {
    int uerr = 0;
    st = cuda_check(ctx, cudaMemcpy(&uerr, ctx->umma_err, sizeof(int), cudaMemcpyDeviceToHost), "umma flag");
    if (st != MLS_OK) return st;
    if (uerr) {
      cudaMemset(ctx->umma_err, 0, sizeof(int));
      return fail(ctx, MLS_ETIMEOUT, "tensor-core trailing update: a bounded wait gave up");
    }
  }
  if (info != 0) return fail(ctx, MLS_ECHOL, "matrix is not positive definite (pivot " + std::to_string(info - 1) + ")");
  return MLS_OK;
}

mls_status factor_dense(mls_ctx* ctx, double* A, int r, double* Acopy, void* W, void* WT) {
  return ctx->opt.precision == MLS_FP64 ? factor_dense_t<double>(ctx, A, r, Acopy, W, WT)
                                        : factor_dense_t<float>(ctx, A, r, Acopy, W, WT);
}

// A = A0 + sigma diag(A0) from the saved operator A0 (row-major r x r)
__global__ void k_shift_restore(double* __restrict__ A, const double* __restrict__ A0, int r, double sigma) {
  const int64_t nn = (int64_t)r * r;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (int64_t)gridDim.x * blockDim.x) {
    const double a = A0[i];
    A[i] = (i / r == i % r) ? a + sigma * fmax(a, 0.0) : a;
  }
}

template <typename VT>
static mls_status factor_t(mls_ctx* ctx) {
  const int r = 12 * ctx->basis.m;
  mls_status st = factor_dense_t<VT>(ctx, ctx->Ac, r, ctx->Acopy, ctx->Linv, ctx->LinvT);
  ctx->coarse_sigma = 0.0;
  double sigma = kShiftFirst;
  for (int k = 0; st == MLS_ECHOL && k < kShiftTries; ++k, sigma *= kShiftGrowth) {
    const int nb = (int)std::min<int64_t>(((int64_t)r * r + kBlock - 1) / kBlock, 4096);
    { ++ctx->launches; k_shift_restore<<<nb, kBlock, 0, ctx->stream>>>(ctx->Ac, ctx->Acopy, r, sigma); }
    if ((st = cuda_check(ctx, cudaGetLastError(), "k_shift_restore")) != MLS_OK) return st;
    ctx->coarse_shift_count++;
    ctx->coarse_sigma = sigma;
    // Acopy keeps the unshifted operator
    st = factor_dense_t<VT>(ctx, ctx->Ac, r, nullptr, ctx->Linv, ctx->LinvT);
  }
  if (st == MLS_OK) {
    const int T = (r + kGramTile - 1) / kGramTile;
    { ++ctx->launches; k_gram_lower<VT><<<T * (T + 1) / 2, 256, 0, ctx->stream>>>((const VT*)ctx->Linv, r, (VT*)ctx->Ainv); }
    st = cuda_check(ctx, cudaGetLastError(), "k_gram_lower");
  }
  ctx->coarse_ready = (st == MLS_OK);
  ctx->coarse_age_steps = 0;
  ctx->coarse_stale = false;
  ctx->coarse_ref_pending = true;
  if (st == MLS_ECHOL) return fail(ctx, MLS_ECHOL, "coarse operator U^T H U: " + ctx->err);
  return st;
}

// y = W^T (W x) with a dense inverse factor pair, solve precision
mls_status dense_apply(mls_ctx* ctx, const void* W, const void* WT, int r, const void* x, void* tmp, void* y) {
  const int nb = trigemv_blocks(r);
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_trigemv<double><<<nb, kBlock, 0, ctx->stream>>>((const double*)W, r, 1, (const double*)x, (double*)tmp, nullptr); }
    { ++ctx->launches; k_trigemv<double><<<nb, kBlock, 0, ctx->stream>>>((const double*)WT, r, 0, (const double*)tmp, (double*)y, nullptr); }
  } else {
    { ++ctx->launches; k_trigemv<float><<<nb, kBlock, 0, ctx->stream>>>((const float*)W, r, 1, (const float*)x, (float*)tmp, nullptr); }
    { ++ctx->launches; k_trigemv<float><<<nb, kBlock, 0, ctx->stream>>>((const float*)WT, r, 0, (const float*)tmp, (float*)y, nullptr); }
  }
  return cuda_check(ctx, cudaGetLastError(), "dense apply");
}

mls_status build_galerkin(mls_ctx* ctx) {
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  switch (ctx->opt.precision) {
    case MLS_FP64: return galerkin_t<double, double>(ctx);
    case MLS_MIXED_FP32: return galerkin_t<double, float>(ctx);
    default: return galerkin_t<double, __nv_bfloat16>(ctx);
  }
}

// ---- Alg. 2's subspace PCG (the paper's literal subspace solve) ---------------------------
// (U^T H U) q = b by conjugate gradient with the 12 x 12 block-Jacobi
// preconditioner (one block per handle, Sec. 3.7.1) and the matrix-free
// product U^T (H (U p)), which runs through the prolongation, the sparse
// product and the restriction kernels; the short coarse vectors (length
// r = 12 m) are updated by one block in float64.

// inverse of each handle's 12 x 12 diagonal block of the dense coarse
// operator (row-major r x r) by Gauss-Jordan elimination with partial
// pivoting, one thread per handle; a zero pivot leaves the identity block
__global__ void k_block_jacobi12(const double* __restrict__ A, int r, double* __restrict__ Binv) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (12 * j >= r) return;
  double a[12][24];
  for (int i = 0; i < 12; ++i)
    for (int k = 0; k < 12; ++k) {
      a[i][k] = A[(int64_t)(12 * j + i) * r + 12 * j + k];
      a[i][12 + k] = (i == k) ? 1.0 : 0.0;
    }
  bool ok = true;
  for (int c = 0; c < 12 && ok; ++c) {
    int piv = c;
    for (int i = c + 1; i < 12; ++i)
      if (fabs(a[i][c]) > fabs(a[piv][c])) piv = i;
    if (!(fabs(a[piv][c]) > 0.0)) { ok = false; break; }
    if (piv != c)
      for (int k = 0; k < 24; ++k) { const double t = a[c][k]; a[c][k] = a[piv][k]; a[piv][k] = t; }
    const double inv = 1.0 / a[c][c];
    for (int k = 0; k < 24; ++k) a[c][k] *= inv;
    for (int i = 0; i < 12; ++i) {
      if (i == c) continue;
      const double f = a[i][c];
      if (f != 0.0)
        for (int k = 0; k < 24; ++k) a[i][k] -= f * a[c][k];
    }
  }
  double* B = Binv + (int64_t)j * 144;
  for (int i = 0; i < 12; ++i)
    for (int k = 0; k < 12; ++k) B[i * 12 + k] = ok ? a[i][12 + k] : (i == k ? 1.0 : 0.0);
}

struct SmsCg {
  double rz, bb, tol2;
  int iter, max_iter, done;  // done: 1 converged, 2 iteration cap, 3 breakdown
};

// z = blockdiag(Binv) res, r entries, one block; returns res.z and res.res
// reduced over the block (valid in thread 0)
__device__ __forceinline__ void sms_precond(int r, const double* __restrict__ Binv, const double* res, double* z) {
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const int j = i / 12, a = i % 12;
    const double* B = Binv + (int64_t)j * 144 + a * 12;
    double s = 0.0;
    for (int k = 0; k < 12; ++k) s += B[k] * res[12 * j + k];
    z[i] = s;
  }
}

__device__ __forceinline__ double block_dot(const double* a, const double* b, int r, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < r; i += blockDim.x) s += a[i] * b[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];  // same order in every thread
  return t;
}

// init: q = 0, res = b, z = B^{-1} res, p = z (and its solve-precision copy)
template <typename VT>
__global__ void __launch_bounds__(256) k_sms_init(int r, const VT* __restrict__ b, const double* __restrict__ Binv,
                                                  double rtol, int max_iter, double* __restrict__ q,
                                                  double* __restrict__ res, double* __restrict__ z,
                                                  double* __restrict__ p, VT* __restrict__ pv, SmsCg* __restrict__ C,
                                                  PcgScalars* __restrict__ S) {
  __shared__ double sh[8];
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    q[i] = 0.0;
    res[i] = (double)b[i];
  }
  __syncthreads();
  sms_precond(r, Binv, res, z);
  __syncthreads();
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    p[i] = z[i];
    pv[i] = (VT)z[i];
  }
  const double rz = block_dot(res, z, r, sh);
  const double bb = block_dot(res, res, r, sh);
  if (threadIdx.x == 0) {
    C->rz = rz;
    C->bb = bb;
    C->tol2 = rtol * rtol * bb;
    C->iter = 0;
    C->max_iter = max_iter;
    C->done = (bb == 0.0) ? 1 : (!(rz > 0.0) || !isfinite(rz) ? 3 : 0);
    S->done = C->done;  // the product kernels skip work once the solve is done
  }
}

template <typename VT>
__global__ void k_cast_coarse(int r, const double* __restrict__ a, VT* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) b[i] = (VT)a[i];
}

// one CG step once s = (U^T H U) p is in sn (solve precision)
template <typename VT>
__global__ void __launch_bounds__(256) k_sms_step(int r, const VT* __restrict__ sn, const double* __restrict__ Binv,
                                                  double* __restrict__ q, double* __restrict__ res,
                                                  double* __restrict__ z, double* __restrict__ p,
                                                  VT* __restrict__ pv, SmsCg* __restrict__ C,
                                                  PcgScalars* __restrict__ S) {
  __shared__ double sh[8];
  __shared__ int s_done;
  if (threadIdx.x == 0) s_done = C->done;
  __syncthreads();
  if (s_done) return;
  double ps = 0.0;  // p . (U^T H U) p
  for (int i = threadIdx.x; i < r; i += blockDim.x) ps += p[i] * (double)sn[i];
  for (int o = 16; o > 0; o >>= 1) ps += __shfl_xor_sync(0xffffffffu, ps, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = ps;
  __syncthreads();
  double pq = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) pq += sh[w];
  const double rz = C->rz;
  if (!(pq > 0.0) || !isfinite(pq)) {
    if (threadIdx.x == 0) { C->done = 3; S->done = 3; }
    return;
  }
  const double alpha = rz / pq;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    q[i] += alpha * p[i];
    res[i] -= alpha * (double)sn[i];
  }
  __syncthreads();
  const double rr = block_dot(res, res, r, sh);
  sms_precond(r, Binv, res, z);
  __syncthreads();
  const double rzn = block_dot(res, z, r, sh);
  const double beta = rzn / rz;
  for (int i = threadIdx.x; i < r; i += blockDim.x) {
    const double pn = z[i] + beta * p[i];
    p[i] = pn;
    pv[i] = (VT)pn;
  }
  if (threadIdx.x == 0) {
    C->rz = rzn;
    C->iter += 1;
    int d = 0;
    if (!isfinite(rr)) d = 3;
    else if (rr <= C->tol2) d = 1;
    else if (!(rzn > 0.0)) d = 3;
    else if (C->iter >= C->max_iter) d = 2;
    C->done = d;
    S->done = d;
  }
}

template <typename VT>
static mls_status sms_pcg_t(mls_ctx* ctx, const void* b, double rtol, int max_iter, int* iters) {
  const int r = 12 * ctx->basis.m;
  mls_status st;
  if (!ctx->sms_buf) {
    if ((st = dalloc(ctx, (void**)&ctx->sms_buf, sizeof(double) * (size_t)r * (4 + 12))) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->sms_cg, sizeof(SmsCg) + sizeof(PcgScalars))) != MLS_OK) return st;
  }
  double* q = ctx->sms_buf;
  double* res = q + r;
  double* z = res + r;
  double* p = z + r;
  double* Binv = p + r;  // [m][144]
  SmsCg* C = (SmsCg*)ctx->sms_cg;
  PcgScalars* S = (PcgScalars*)((char*)ctx->sms_cg + sizeof(SmsCg));
  { ++ctx->launches; k_block_jacobi12<<<(ctx->basis.m + 63) / 64, 64, 0, ctx->stream>>>(ctx->Acopy, r, Binv); }
  VT* pv = (VT*)ctx->cvec2;
  VT* sn = (VT*)ctx->cvec;
  { ++ctx->launches; k_sms_init<VT><<<1, 256, 0, ctx->stream>>>(r, (const VT*)b, Binv, rtol, max_iter, q, res, z, p, pv, C, S); }
  if ((st = cuda_check(ctx, cudaGetLastError(), "k_sms_init")) != MLS_OK) return st;
  const BasisView BV = basis_view(ctx);
  const dim3 rgrid(restrict_blocks(ctx->basis.nrchunk)), rblock(32 * kRestrictWarps);
  const int chunk = 8;
  SmsCg h{};
  for (int it = 0; it < max_iter; it += chunk) {
    for (int c = 0; c < chunk; ++c) {
      // w = U p, y = H w, sn = U^T y = (U^T H U) p
      { ++ctx->launches; k_prolong<VT><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(BV, pv, nullptr, nullptr, nullptr,
                                                                                   VT(0), (Vec4<VT>*)ctx->vp, S); }
      if ((st = launch_spmv(ctx, ctx->vp, ctx->vq)) != MLS_OK) return st;
      { ++ctx->launches; k_restrict<VT><<<rgrid, rblock, 0, ctx->stream>>>(BV, (const Vec4<VT>*)ctx->vq, sn, S); }
      { ++ctx->launches; k_sms_step<VT><<<1, 256, 0, ctx->stream>>>(r, sn, Binv, q, res, z, p, pv, C, S); }
    }
    if ((st = cuda_check(ctx, cudaMemcpyAsync(&h, C, sizeof(SmsCg), cudaMemcpyDeviceToHost, ctx->stream), "sms state")) != MLS_OK)
      return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sms sync")) != MLS_OK) return st;
    if (h.done) break;
  }
  *iters = h.iter;
  if (h.done == 3) return fail(ctx, MLS_ENONFINITE, "subspace PCG breakdown");
  // the solution, in solve precision, into cvec
  { ++ctx->launches; k_cast_coarse<VT><<<(r + 255) / 256, 256, 0, ctx->stream>>>(r, q, (VT*)ctx->cvec); }
  return cuda_check(ctx, cudaGetLastError(), "sms solution");
}

// M = A T (A = U^T H U, row-major r x r; T the SMS coordinates of an affine
// motion about o_a): for row i and component c, M[i][4c] = sum_j A[i][12j+4c]
// and M[i][4c+l] = sum_j (A[i][12j+4c+l] + d_jl A[i][12j+4c]), d_j = o_j - o_a
__global__ void k_affine_mt(const double* __restrict__ A, int r, int m, const double* __restrict__ origins,
                            double o0, double o1, double o2, double* __restrict__ M) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= 3 * r) return;
  const int i = idx / 3, c = idx % 3;
  const double* a = A + (int64_t)i * r;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  for (int j = 0; j < m; ++j) {
    const double a0 = a[12 * j + 4 * c];
    s0 += a0;
    s1 += a[12 * j + 4 * c + 1] + (origins[3 * j] - o0) * a0;
    s2 += a[12 * j + 4 * c + 2] + (origins[3 * j + 1] - o1) * a0;
    s3 += a[12 * j + 4 * c + 3] + (origins[3 * j + 2] - o2) * a0;
  }
  double* out = M + (int64_t)i * 12 + 4 * c;
  out[0] = s0; out[1] = s1; out[2] = s2; out[3] = s3;
}

mls_status affine_operator(mls_ctx* ctx, const double om[3]) {
  const int m = ctx->basis.m, r = 12 * m;
  mls_status st;
  if (!ctx->sms_m && (st = dalloc(ctx, (void**)&ctx->sms_m, sizeof(double) * (size_t)r * 12)) != MLS_OK) return st;
  { ++ctx->launches; k_affine_mt<<<(3 * r + 127) / 128, 128, 0, ctx->stream>>>(ctx->Acopy, r, m, ctx->basis.origins,
                                                                              om[0], om[1], om[2], ctx->sms_m); }
  return cuda_check(ctx, cudaGetLastError(), "k_affine_mt");
}

// U^T H U into Ac and its copy Acopy, without a factorisation (the literal
// subspace solve of direction 2 needs the operator's blocks, not a factor)
mls_status build_coarse_unfactored(mls_ctx* ctx) {
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "assemble H before building the coarse operator");
  const int r = 12 * ctx->basis.m;
  int tk = prof_begin(ctx, MLS_PROF_GALERKIN);
  mls_status st;
  if (ctx->cub_scale && (st = launch_assemble_cubature(ctx, ctx->xk)) != MLS_OK) return st;
  if ((st = build_galerkin(ctx)) != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->Acopy, ctx->Ac, sizeof(double) * r * r, cudaMemcpyDeviceToDevice,
                                       ctx->stream), "A copy");
  prof_end(ctx, tk);
  ctx->galerkin_ready = (st == MLS_OK);
  ctx->coarse_ready = false;
  return st;
}

// (U^T H U) q = b (b: [r] coarse vector in solve precision) by Alg. 2's
// subspace PCG to relative residual rtol; the operator's diagonal blocks come
// from the Galerkin product's unfactored copy (Acopy).  The solution lands in
// cvec (solve precision); the full-space vectors vp and vq are scratch.
mls_status sms_pcg(mls_ctx* ctx, const void* b, double rtol, int max_iter, int* iters) {
  return ctx->opt.precision == MLS_FP64 ? sms_pcg_t<double>(ctx, b, rtol, max_iter, iters)
                                        : sms_pcg_t<float>(ctx, b, rtol, max_iter, iters);
}

// ---- damping of the block-Jacobi smoother ------------------------------------------------
// The symmetric two-level cycle (pre- and post-smoothing with omega D^{-1},
// D the 3x3 block diagonal of H) is positive definite if and only if
// omega lambda_max(D^{-1} H) < 2.  With omega = 0 the library takes
// omega = kOmegaFrac * 2 / theta, theta the largest Ritz value of
// kLanczosSteps Lanczos steps on C^T H C, where D^{-1} = C C^T per vertex:
// C^T H C is symmetric and similar to D^{-1} H, and a Ritz value never
// exceeds lambda_max, so kOmegaFrac is the margin to the limit.
constexpr double kOmegaFrac = 0.9;

// C with C C^T = D^{-1} (lower, row-major 3x3) from the stored D^{-1} block;
// a non-positive pivot zeroes the rest of the factor
template <typename VT>
__device__ __forceinline__ void dinv_factor(const VT* __restrict__ A, VT (&C)[9]) {
  const VT a00 = A[0], a10 = A[3], a11 = A[4], a20 = A[6], a21 = A[7], a22 = A[8];
  const VT l00 = a00 > VT(0) ? sqrt(a00) : VT(0);
  const VT l10 = l00 > VT(0) ? a10 / l00 : VT(0), l20 = l00 > VT(0) ? a20 / l00 : VT(0);
  const VT d11 = a11 - l10 * l10;
  const VT l11 = d11 > VT(0) ? sqrt(d11) : VT(0);
  const VT l21 = l11 > VT(0) ? (a21 - l20 * l10) / l11 : VT(0);
  const VT d22 = a22 - l20 * l20 - l21 * l21;
  const VT l22 = d22 > VT(0) ? sqrt(d22) : VT(0);
  C[0] = l00; C[1] = VT(0); C[2] = VT(0);
  C[3] = l10; C[4] = l11; C[5] = VT(0);
  C[6] = l20; C[7] = l21; C[8] = l22;
}

// starting vector: a fixed hash of the component index in [-1, 1]; |w|^2
// into beta[0] (as its square root)
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_lz_seed(int n, Vec4<VT>* __restrict__ w, GridReduce gr,
                                                    double* __restrict__ beta) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < n) {
    VT c[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      unsigned h = (unsigned)(3 * v + k) * 2654435761u;  // multiplicative hash, then xorshift mixing
      h ^= h >> 16; h *= 2246822519u; h ^= h >> 13; h *= 3266489917u; h ^= h >> 16;
      c[k] = VT((double)h * (2.0 / 4294967295.0) - 1.0);
      acc[0] += (double)c[k] * c[k];
    }
    w[v] = Vec4<VT>{c[0], c[1], c[2], VT(0)};
  }
  if (grid_sum<1>(acc, gr, RS_MISC) && threadIdx.x == 0) beta[0] = sqrt(acc[0]);
}

// v = w / beta[j] (in place) and t = C v
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_lz_scale(int n, const VT* __restrict__ dinv, Vec4<VT>* __restrict__ wv,
                                                     const double* __restrict__ beta, int j, Vec4<VT>* __restrict__ t) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double b = beta[j];
  const VT s = b > 0.0 ? VT(1.0 / b) : VT(0);
  const Vec4<VT> x = wv[v];
  const VT x0 = s * x.x, x1 = s * x.y, x2 = s * x.z;
  wv[v] = Vec4<VT>{x0, x1, x2, VT(0)};
  VT C[9];
  dinv_factor<VT>(dinv + (int64_t)v * 9, C);
  t[v] = Vec4<VT>{C[0] * x0, C[3] * x0 + C[4] * x1, C[6] * x0 + C[7] * x1 + C[8] * x2, VT(0)};
}

// alpha[j] = t . y  (= v^T C^T H C v)
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_lz_alpha(int n, const Vec4<VT>* __restrict__ t, const Vec4<VT>* __restrict__ y,
                                                     GridReduce gr, double* __restrict__ alpha, int j) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < n) {
    const Vec4<VT> a = t[v], b = y[v];
    acc[0] = (double)a.x * b.x + (double)a.y * b.y + (double)a.z * b.z;
  }
  if (grid_sum<1>(acc, gr, RS_MISC) && threadIdx.x == 0) alpha[j] = acc[0];
}

// w = C^T y - alpha[j] v - beta[j] v_prev, written over v_prev (j > 0; for
// j = 0 the last term is absent); |w| into beta[j + 1]
template <typename VT>
__global__ void __launch_bounds__(kBlock) k_lz_residual(int n, const VT* __restrict__ dinv, const Vec4<VT>* __restrict__ y,
                                                        const Vec4<VT>* __restrict__ vc, Vec4<VT>* __restrict__ vp,
                                                        const double* __restrict__ alpha,
                                                        const double* __restrict__ beta, int j, GridReduce gr,
                                                        double* __restrict__ beta_out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < n) {
    VT C[9];
    dinv_factor<VT>(dinv + (int64_t)v * 9, C);
    const Vec4<VT> yy = y[v], x = vc[v];
    const VT a = (VT)alpha[j], b = j > 0 ? (VT)beta[j] : VT(0);
    const Vec4<VT> xp = j > 0 ? vp[v] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
    const VT w0 = C[0] * yy.x + C[3] * yy.y + C[6] * yy.z - a * x.x - b * xp.x;
    const VT w1 = C[4] * yy.y + C[7] * yy.z - a * x.y - b * xp.y;
    const VT w2 = C[8] * yy.z - a * x.z - b * xp.z;
    vp[v] = Vec4<VT>{w0, w1, w2, VT(0)};
    acc[0] = (double)w0 * w0 + (double)w1 * w1 + (double)w2 * w2;
  }
  if (grid_sum<1>(acc, gr, RS_MISC) && threadIdx.x == 0) beta_out[j + 1] = sqrt(acc[0]);
}

template <typename VT>
static mls_status lanczos_t(mls_ctx* ctx, double* alpha_h, double* beta_h) {
  const int n = ctx->n;
  const int nb = nblk(n);
  const VT* dinv = (const VT*)ctx->dinv;
  Vec4<VT>* buf[2] = {(Vec4<VT>*)ctx->vp, (Vec4<VT>*)ctx->vq};  // v_j and v_{j-1} / w, alternating
  Vec4<VT>* t = (Vec4<VT>*)ctx->vw;
  Vec4<VT>* y = (Vec4<VT>*)ctx->vz2;
  double* alpha = ctx->lz;
  double* beta = ctx->lz + kLanczosSteps;
  { ++ctx->launches; k_lz_seed<VT><<<nb, kBlock, 0, ctx->stream>>>(n, buf[0], ctx->red, beta); }
  int cur = 0;
  for (int j = 0; j < kLanczosSteps; ++j) {
    { ++ctx->launches; k_lz_scale<VT><<<nb, kBlock, 0, ctx->stream>>>(n, dinv, buf[cur], beta, j, t); }
    mls_status st = launch_spmv(ctx, t, y);
    if (st != MLS_OK) return st;
    { ++ctx->launches; k_lz_alpha<VT><<<nb, kBlock, 0, ctx->stream>>>(n, t, y, ctx->red, alpha, j); }
    { ++ctx->launches; k_lz_residual<VT><<<nb, kBlock, 0, ctx->stream>>>(n, dinv, y, buf[cur], buf[cur ^ 1], alpha,
                                                                      beta, j, ctx->red, beta); }
    cur ^= 1;
  }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "lanczos");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(alpha_h, alpha, sizeof(double) * kLanczosSteps, cudaMemcpyDeviceToHost, ctx->stream),
                  "lanczos readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(beta_h, beta, sizeof(double) * (kLanczosSteps + 1), cudaMemcpyDeviceToHost,
                                       ctx->stream), "lanczos readback");
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "lanczos sync");
}

// omega_eff from the Lanczos estimate (opt.omega = 0), else opt.omega
static mls_status choose_omega(mls_ctx* ctx) {
  if (ctx->opt.omega > 0.0) {
    ctx->omega_eff = ctx->opt.omega;
    return MLS_OK;
  }
  double a[kLanczosSteps], b[kLanczosSteps + 1];
  mls_status st = ctx->opt.precision == MLS_FP64 ? lanczos_t<double>(ctx, a, b) : lanczos_t<float>(ctx, a, b);
  if (st != MLS_OK) return st;
  // b[0] normalises the start vector; T_k has diagonal a[0..k-1] and
  // off-diagonal b[1..k-1].  Stop at an invariant subspace or a bad value.
  int k = 0;
  while (k < kLanczosSteps && std::isfinite(a[k]) && std::isfinite(b[k]) && b[k] > 0.0) {
    ++k;
    if (!(b[k] > 1e-12 * std::fabs(a[k - 1]))) break;
  }
  if (k == 0) return fail(ctx, MLS_ENONFINITE, "smoother damping: Lanczos estimate failed");
  const double theta = tridiag_max_eig(a, b + 1, k);
  if (!(theta > 0.0) || !std::isfinite(theta)) return fail(ctx, MLS_ENONFINITE, "smoother damping: bad estimate");
  ctx->omega_lmax = theta;
  ctx->omega_eff = std::min(1.0, kOmegaFrac * 2.0 / theta);
  return MLS_OK;
}

mls_status build_coarse(mls_ctx* ctx) {
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "assemble H before building the coarse operator");
  mls_status st;
  if ((st = choose_omega(ctx)) != MLS_OK) return st;
  int tk = prof_begin(ctx, MLS_PROF_GALERKIN);
  if (ctx->cub_scale && (st = launch_assemble_cubature(ctx, ctx->xk)) != MLS_OK) return st;
  st = build_galerkin(ctx);
  if (st != MLS_OK) return st;
  prof_end(ctx, tk);
  tk = prof_begin(ctx, MLS_PROF_CHOLESKY);
  st = ctx->opt.precision == MLS_FP64 ? factor_t<double>(ctx) : factor_t<float>(ctx);
  prof_end(ctx, tk);
  return st;
}

// c_out = A^{-1} c_in with the dense inverse W^T W (one product; c_out must
// not alias c_in)
template <typename VT>
static mls_status coarse_apply_t(mls_ctx* ctx, const VT* c_in, VT* c_out, const PcgScalars* S) {
  const int r = 12 * ctx->basis.m;
  const int nb = trigemv_blocks(r);
  ++ctx->launches;
  return cuda_check(ctx, launch_chained(k_trigemv<VT>, dim3(nb), dim3(kBlock), ctx->stream, (const VT*)ctx->Ainv, r, 2,
                                        c_in, c_out, S), "coarse product");
}

mls_status coarse_apply(mls_ctx* ctx, const void* c_in, void* c_out) {
  if (!ctx->coarse_ready) return fail(ctx, MLS_EINVAL, "coarse operator not built");
  if (c_in == c_out) return fail(ctx, MLS_EINVAL, "coarse_apply: output must not alias the input");
  if (ctx->opt.precision == MLS_FP64) return coarse_apply_t<double>(ctx, (const double*)c_in, (double*)c_out, nullptr);
  return coarse_apply_t<float>(ctx, (const float*)c_in, (float*)c_out, nullptr);
}

template <typename VT>
static mls_status two_level_t(mls_ctx* ctx, const Vec4<VT>* r, Vec4<VT>* z, const PcgScalars* S) {
  const BasisView BV = basis_view(ctx);
  const VT omega = (VT)ctx->omega_eff;
  VT* c = (VT*)ctx->cvec;
  const VT* dinv = (const VT*)ctx->dinv;
  if (ctx->opt.cycle == MLS_CYCLE_ADDITIVE) {
    { ++ctx->launches; k_restrict<VT><<<restrict_blocks(ctx->basis.nrchunk), 32 * kRestrictWarps, 0, ctx->stream>>>(BV, r, c, S); }
    VT* c2 = (VT*)ctx->cvec2;
    mls_status st = coarse_apply_t<VT>(ctx, c, c2, S);
    if (st != MLS_OK) return st;
    { ++ctx->launches; k_prolong<VT><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(BV, c2, nullptr, dinv, r, omega, z, S); }
    return cuda_check(ctx, cudaGetLastError(), "two-level additive");
  }
  // multiplicative: z1 = S r; t = r - H z1; z2 = z1 + Q t; t = r - H z2; z = z2 + S t
  Vec4<VT>* tmp = (Vec4<VT>*)ctx->vw;
  mls_status st = launch_jacobi(ctx, r, z, ctx->omega_eff, S);
  if (st != MLS_OK) return st;
  if ((st = launch_residual(ctx, r, z, tmp, S)) != MLS_OK) return st;
  { ++ctx->launches; k_restrict<VT><<<restrict_blocks(ctx->basis.nrchunk), 32 * kRestrictWarps, 0, ctx->stream>>>(BV, tmp, c, S); }
  if ((st = coarse_apply_t<VT>(ctx, c, (VT*)ctx->cvec2, S)) != MLS_OK) return st;
  { ++ctx->launches; k_prolong<VT><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(BV, (const VT*)ctx->cvec2, z, nullptr, nullptr, omega, z, S); }
  if ((st = launch_residual(ctx, r, z, tmp, S)) != MLS_OK) return st;
  { ++ctx->launches; k_prolong<VT><<<prolong_blocks(ctx->n), kBlock, 0, ctx->stream>>>(BV, nullptr, z, dinv, tmp, omega, z, S); }
  return cuda_check(ctx, cudaGetLastError(), "two-level multiplicative");
}

mls_status launch_post_smooth_rz(mls_ctx* ctx, const void* r, const void* z2, void* zout, int first, int it,
                                 PcgScalars* S);

// One application of the two-level cycle inside PCG, with z1 = omega D^{-1} r
// already in place: additive z = z1 + U A^{-1} U^T r; multiplicative
// z2 = z1 + U A^{-1} U^T (r - H z1), zf = z2 + omega D^{-1} (r - H z2).  Ends
// with r.zf and beta.
template <typename VT>
static mls_status two_level_step_t(mls_ctx* ctx, const Vec4<VT>* r, Vec4<VT>* z1, Vec4<VT>* zf, int first, int it,
                                   PcgScalars* S) {
  const BasisView BV = basis_view(ctx);
  VT* c = (VT*)ctx->cvec;
  mls_status st;
  const dim3 rgrid(restrict_blocks(ctx->basis.nrchunk)), rblock(32 * kRestrictWarps);
  if (ctx->opt.cycle == MLS_CYCLE_ADDITIVE) {
    ++ctx->launches;
    if ((st = cuda_check(ctx, launch_chained(k_restrict<VT>, rgrid, rblock, ctx->stream, BV, r, c, S), "k_restrict")) != MLS_OK)
      return st;
    if ((st = coarse_apply_t<VT>(ctx, c, (VT*)ctx->cvec2, S)) != MLS_OK) return st;
    ++ctx->launches;
    return cuda_check(ctx, launch_chained(k_prolong_rz<VT>, dim3(nblk(ctx->n)), dim3(kBlock), ctx->stream, BV,
                                          (const VT*)ctx->cvec2, r, z1, first, it, ctx->red, ctx->pcg_fix, S),
                      "k_prolong_rz");
  }
  Vec4<VT>* tmp = (Vec4<VT>*)ctx->vw;
  if ((st = launch_residual(ctx, r, z1, tmp, S)) != MLS_OK) return st;
  ++ctx->launches;
  if ((st = cuda_check(ctx, launch_chained(k_restrict<VT>, rgrid, rblock, ctx->stream, BV, (const Vec4<VT>*)tmp, c, S),
                       "k_restrict")) != MLS_OK)
    return st;
  if ((st = coarse_apply_t<VT>(ctx, c, (VT*)ctx->cvec2, S)) != MLS_OK) return st;
  ++ctx->launches;
  if ((st = cuda_check(ctx, launch_chained(k_prolong<VT>, dim3(prolong_blocks(ctx->n)), dim3(kBlock), ctx->stream, BV, (const VT*)ctx->cvec2,
                                           (const Vec4<VT>*)z1, (const VT*)nullptr, (const Vec4<VT>*)nullptr, VT(0), z1,
                                           S), "k_prolong")) != MLS_OK)
    return st;
  return launch_post_smooth_rz(ctx, r, z1, zf, first, it, S);
}

mls_status two_level_pcg_step(mls_ctx* ctx, const void* r, void* z1, void* zf, int first, int it, PcgScalars* S) {
  if (ctx->opt.precision == MLS_FP64)
    return two_level_step_t<double>(ctx, (const Vec4d*)r, (Vec4d*)z1, (Vec4d*)zf, first, it, S);
  return two_level_step_t<float>(ctx, (const Vec4f*)r, (Vec4f*)z1, (Vec4f*)zf, first, it, S);
}

mls_status precond_apply_dev(mls_ctx* ctx, const void* r, void* z, const PcgScalars* S) {
  if (ctx->opt.preconditioner == MLS_PRECOND_BLOCK_JACOBI) return launch_jacobi(ctx, r, z, 1.0, S);
  if (!ctx->coarse_ready) return fail(ctx, MLS_EINVAL, "two-level preconditioner needs the coarse operator");
  if (ctx->opt.precision == MLS_FP64) return two_level_t<double>(ctx, (const Vec4d*)r, (Vec4d*)z, S);
  return two_level_t<float>(ctx, (const Vec4f*)r, (Vec4f*)z, S);
}

}  // namespace mls
