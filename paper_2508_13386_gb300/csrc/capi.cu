// C ABI: context management, mesh/basis upload and the Newton timestep driver
// (Sec. 3.1 implicit Euler on Eq. IP; Eq. 5 linear solves; Sec. 3.9 filtered
// backtracking line search).  The driver keeps every vector on the device and
// reads back only the few scalars that steer the loop (PCG convergence flags,
// step norms, line-search energies).
#include "mls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

using namespace mls;

namespace mls {

mls_status fail(mls_ctx* ctx, mls_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

mls_status cuda_check(mls_ctx* ctx, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MLS_OK;
  return fail(ctx, MLS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

mls_status dalloc(mls_ctx* ctx, void** p, size_t bytes) {
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(ctx, MLS_ENOMEM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  }
  ctx->allocs.push_back(q);
  *p = q;
  return MLS_OK;
}

void dfree(mls_ctx* ctx, void* p) {
  if (!p) return;
  auto it = std::find(ctx->allocs.begin(), ctx->allocs.end(), p);
  if (it != ctx->allocs.end()) ctx->allocs.erase(it);
  cudaFree(p);
}

int solve_bytes(const mls_ctx* ctx) { return ctx->opt.precision == MLS_FP64 ? 8 : 4; }
int storage_bytes(const mls_ctx* ctx) {
  return ctx->opt.precision == MLS_FP64 ? 8 : (ctx->opt.precision == MLS_MIXED_FP32 ? 4 : 2);
}
int element_bytes(const mls_ctx* ctx) { return ctx->opt.precision == MLS_FP64 ? 8 : 4; }

// g . d over float64 vertex vectors
__global__ void __launch_bounds__(kBlock) k_dot4(int n, const Vec4d* __restrict__ a, const Vec4d* __restrict__ b,
                                                 GridReduce gr, double* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < n) {
    const Vec4d x = a[v], y = b[v];
    acc[0] = x.x * y.x + x.y * y.y + x.z * y.z;
  }
  if (grid_sum<1>(acc, gr, RS_MISC) && threadIdx.x == 0) *out = acc[0];
}

static mls_status read_scalar(mls_ctx* ctx, const double* dev, double* host_out);

// sum over vertices of |d_v|_2 (float64)
__global__ void k_vnorm_sum(int n, const Vec4d* __restrict__ d, GridReduce gr, double* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < n) {
    const Vec4d a = d[v];
    acc[0] = sqrt(a.x * a.x + a.y * a.y + a.z * a.z);
  }
  if (grid_sum<1>(acc, gr, RS_MISC) && threadIdx.x == 0) *out = acc[0];
}

static mls_status vnorm_sum(mls_ctx* ctx, const Vec4d* d, double* out) {
  const int nb = (ctx->n + kBlock - 1) / kBlock;
  { ++ctx->launches; k_vnorm_sum<<<nb, kBlock, 0, ctx->stream>>>(ctx->n, d, ctx->red, ctx->dscal + 9); }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "k_vnorm_sum");
  if (st != MLS_OK) return st;
  return read_scalar(ctx, ctx->dscal + 9, out);
}

static mls_status dot4(mls_ctx* ctx, const Vec4d* a, const Vec4d* b, double* out) {
  const int nb = (ctx->n + kBlock - 1) / kBlock;
  { ++ctx->launches; k_dot4<<<nb, kBlock, 0, ctx->stream>>>(ctx->n, a, b, ctx->red, ctx->dscal + 8); }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "k_dot4");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 8, ctx->dscal + 8, sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream), "dot readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "dot sync");
  *out = ctx->dscal_host[8];
  return st;
}

static mls_status read_scalar(mls_ctx* ctx, const double* dev, double* host_out) {
  mls_status st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 10, dev, sizeof(double),
                                                  cudaMemcpyDeviceToHost, ctx->stream), "scalar readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "scalar sync");
  *host_out = ctx->dscal_host[10];
  return st;
}

int prof_begin(mls_ctx* ctx, int cls) {
  if (!(ctx->prof_mask & (1u << cls))) return -1;
  const int base = (int)ctx->prof_pending.size() * 2;
  while ((int)ctx->prof_pool.size() < base + 2) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return -1; }
    ctx->prof_pool.push_back(e);
  }
  cudaEventRecord(ctx->prof_pool[base], ctx->stream);
  ctx->prof_pending.emplace_back(cls, base);
  return base;
}

void prof_end(mls_ctx* ctx, int token) {
  if (token < 0) return;
  cudaEventRecord(ctx->prof_pool[token + 1], ctx->stream);
}

void prof_flush(mls_ctx* ctx) {
  for (auto& pe : ctx->prof_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ctx->prof_pool[pe.second], ctx->prof_pool[pe.second + 1]) == cudaSuccess) {
      ctx->prof_ms[pe.first] += ms;
      ctx->prof_n[pe.first] += 1;
    } else {
      cudaGetLastError();
    }
  }
  ctx->prof_pending.clear();
}

// SELL-32 sparsity of H from the tet adjacency (diagonal block first, then
// ascending columns), with spare[v] (nullable) empty slots after row v's
// blocks, and the per-slot lists of element blocks that assembly sums.
// Replaces the previous pattern arrays.
mls_status build_pattern(mls_ctx* ctx, const std::vector<int>* spare) {
  const int n = ctx->n, t = ctx->t;
  const int* tets = ctx->h_tets.data();
  std::vector<std::vector<int>> nbr(n);
  for (int e = 0; e < t; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) nbr[tets[4 * e + a]].push_back(tets[4 * e + b]);
  std::vector<int> row_len(n);
  for (int v = 0; v < n; ++v) {
    auto& L = nbr[v];
    std::sort(L.begin(), L.end());
    L.erase(std::unique(L.begin(), L.end()), L.end());
    auto it = std::find(L.begin(), L.end(), v);
    if (it == L.end()) L.insert(L.begin(), v);
    else std::rotate(L.begin(), it, it + 1);
    row_len[v] = (int)L.size();
  }
  const int n_slices = (n + kSlice - 1) / kSlice;
  std::vector<int> slice_ptr(n_slices + 1, 0);
  for (int s = 0; s < n_slices; ++s) {
    int w = 0;
    for (int v = s * kSlice; v < std::min(n, (s + 1) * kSlice); ++v)
      w = std::max(w, row_len[v] + (spare ? (*spare)[v] : 0));
    slice_ptr[s + 1] = slice_ptr[s] + w;
  }
  const int64_t n_groups = slice_ptr[n_slices];
  const int64_t n_slots = n_groups * kSlice;
  if (n_slots + 1 > INT32_MAX) return fail(ctx, MLS_EINVAL, "sparsity pattern of H too large");
  std::vector<int> group_slice(n_groups), col(n_slots);
  for (int s = 0; s < n_slices; ++s)
    for (int g = slice_ptr[s]; g < slice_ptr[s + 1]; ++g) group_slice[g] = s;
  int64_t nnzb = 0;
  for (int v = 0; v < n; ++v) {
    const int s = v / kSlice, lane = v % kSlice;
    const int w = slice_ptr[s + 1] - slice_ptr[s];
    for (int k = 0; k < w; ++k)
      col[((int64_t)slice_ptr[s] + k) * kSlice + lane] = k < row_len[v] ? nbr[v][k] : v;
    nnzb += row_len[v];
  }
  // element-block contributions per slot (CSR over slots)
  std::vector<int> asm_cnt(n_slots + 1, 0);
  std::vector<int64_t> code_slot(16 * (size_t)t);
  for (int e = 0; e < t; ++e)
    for (int a = 0; a < 4; ++a) {
      const int v = tets[4 * e + a];
      const auto& L = nbr[v];
      const int s = v / kSlice, lane = v % kSlice;
      for (int b = 0; b < 4; ++b) {
        const int w = tets[4 * e + b];
        const int k = (int)(std::find(L.begin(), L.end(), w) - L.begin());
        const int64_t slot = ((int64_t)slice_ptr[s] + k) * kSlice + lane;
        code_slot[16 * (size_t)e + 4 * a + b] = slot;
        asm_cnt[slot + 1]++;
      }
    }
  for (int64_t s = 0; s < n_slots; ++s) asm_cnt[s + 1] += asm_cnt[s];
  std::vector<int> asm_code(16 * (size_t)t);
  {
    std::vector<int> fill(asm_cnt.begin(), asm_cnt.end() - 1);
    for (int e = 0; e < t; ++e)
      for (int ab = 0; ab < 16; ++ab) asm_code[fill[code_slot[16 * (size_t)e + ab]]++] = 16 * e + ab;
  }
  int** old[] = {&ctx->slice_ptr, &ctx->group_slice, &ctx->col, &ctx->row_len, &ctx->asm_ptr, &ctx->asm_code};
  for (int** p : old) {
    dfree(ctx, *p);
    *p = nullptr;
  }
  auto up = [&](void** dst, const void* src, size_t bytes) -> mls_status {
    mls_status st = dalloc(ctx, dst, bytes);
    if (st != MLS_OK) return st;
    return cuda_check(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "pattern upload");
  };
  mls_status st;
  if ((st = up((void**)&ctx->slice_ptr, slice_ptr.data(), sizeof(int) * (n_slices + 1))) != MLS_OK) return st;
  if ((st = up((void**)&ctx->group_slice, group_slice.data(), sizeof(int) * n_groups)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->col, col.data(), sizeof(int) * n_slots)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->row_len, row_len.data(), sizeof(int) * n)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->asm_ptr, asm_cnt.data(), sizeof(int) * (n_slots + 1))) != MLS_OK) return st;
  if ((st = up((void**)&ctx->asm_code, asm_code.data(), sizeof(int) * 16 * (size_t)t)) != MLS_OK) return st;
  ctx->n_slices = n_slices;
  ctx->n_groups = n_groups;
  ctx->nnzb = nnzb;
  ctx->h_slice_ptr = slice_ptr;
  ctx->h_row_len = row_len;
  ctx->h_col = col;
  return MLS_OK;
}

static void free_all(mls_ctx* ctx) {
  for (void* p : ctx->allocs) cudaFree(p);
  ctx->allocs.clear();
  ctx->Am = nullptr; ctx->Wm = ctx->WmT = ctx->ws_c = ctx->ws_c2 = ctx->ws_tmp = nullptr;
  ctx->ws_hist = ctx->ws_qg = ctx->ws_qtilde = ctx->ws_qnext = nullptr;
  ctx->ws_feat = ctx->ws_target = ctx->ws_pred = nullptr;
  ctx->ws_hsave = nullptr;
  ctx->oz_fwd = nullptr;
  ctx->oz_e = ctx->umma_err = nullptr;
  ctx->sms_buf = nullptr;
  ctx->sms_cg = nullptr;
  ctx->sms_m = nullptr;
  ctx->ehess_lag = ctx->hval_lag = ctx->dinv_lag = nullptr;
  ctx->ws_ready = ctx->ws_enabled = ctx->ws_hist_valid = ctx->ws_record = false;
  ctx->ws_mlp = nullptr;
  ctx->basis = Basis{};
  ctx->has_basis = false;
  ctx->coarse_ready = false;
  ctx->galerkin_ready = false;
  ctx->assembled = false;
  ctx->cub_scale = nullptr;
  ctx->hval_cub = nullptr;
  int* keep = ctx->cs.cnt_host;  // pinned, freed with the context
  ctx->cs = mls::ContactState{};
  ctx->cs.cnt_host = keep;
}

static mls_status alloc_state(mls_ctx* ctx);

}  // namespace mls

extern "C" {

mls_status mls_default_options(mls_options* opt) {
  if (!opt) return MLS_EINVAL;
  opt->precision = MLS_FP64;
  opt->preconditioner = MLS_PRECOND_BLOCK_JACOBI;
  opt->cycle = MLS_CYCLE_ADDITIVE;
  opt->omega = 1.0;
  opt->newton_tol = 1e-10;
  opt->pcg_rtol = 1e-4;
  opt->max_newton = 50;
  opt->max_pcg = 20000;
  opt->coarse_refresh = 0;
  opt->coarse_lag_steps = 0;
  opt->pcg_check_every = 16;
  opt->persistent = 0;
  opt->persist_blocks_per_sm = 0;
  opt->direction = 0;
  opt->refine_iters = 20;
  opt->paper_tol = 1e-3;
  opt->sub_rtol = 1e-4;
  opt->hessian_lag = 0;
  opt->stream = nullptr;
  return MLS_OK;
}

static mls_status check_options(const mls_options* o) {
  if (o->precision < MLS_FP64 || o->precision > MLS_MIXED_BF16) return MLS_EINVAL;
  if (o->preconditioner < 0 || o->preconditioner > 1) return MLS_EINVAL;
  if (o->cycle < 0 || o->cycle > 1) return MLS_EINVAL;
  if (!(o->newton_tol > 0) || !(o->pcg_rtol > 0) || o->max_newton < 1 || o->max_pcg < 1) return MLS_EINVAL;
  if (!(o->omega >= 0.0) || o->coarse_refresh < 0 || o->coarse_lag_steps < 0 || o->pcg_check_every < 1)
    return MLS_EINVAL;
  if (o->persistent < 0 || o->persistent > 1 || o->persist_blocks_per_sm < 0 || o->persist_blocks_per_sm > 32)
    return MLS_EINVAL;
  if (o->direction < 0 || o->direction > 2 || o->refine_iters < 0 || !(o->paper_tol > 0)) return MLS_EINVAL;
  if (o->direction == 2 && !(o->sub_rtol > 0 && o->sub_rtol < 1)) return MLS_EINVAL;
  return MLS_OK;
}

mls_status mls_create(mls_ctx** out, const mls_options* opt) {
  if (!out) return MLS_EINVAL;
  *out = nullptr;
  mls_ctx* ctx = new (std::nothrow) mls_ctx();
  if (!ctx) return MLS_ENOMEM;
  if (opt) {
    if (check_options(opt) != MLS_OK) { delete ctx; return MLS_EINVAL; }
    ctx->opt = *opt;
  } else {
    mls_default_options(&ctx->opt);
  }
  ctx->omega_eff = ctx->opt.omega > 0.0 ? ctx->opt.omega : 0.5;
  ctx->stream = (cudaStream_t)ctx->opt.stream;
  if (cudaGetDevice(&ctx->device) != cudaSuccess) { cudaGetLastError(); delete ctx; return MLS_ECUDA; }
  void* h = nullptr;
  if (cudaMallocHost(&h, sizeof(double) * 16 + sizeof(PcgScalars)) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return MLS_ECUDA;
  }
  ctx->host_allocs.push_back(h);
  ctx->dscal_host = (double*)h;
  ctx->pcg_host = (PcgScalars*)((char*)h + sizeof(double) * 16);
  *out = ctx;
  return MLS_OK;
}

mls_status mls_destroy(mls_ctx* ctx) {
  if (!ctx) return MLS_OK;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  free_all(ctx);
  for (void* p : ctx->host_allocs) cudaFreeHost(p);
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  delete ctx;
  return MLS_OK;
}

const char* mls_last_error(const mls_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

mls_status mls_set_options(mls_ctx* ctx, const mls_options* opt) {
  if (!ctx || !opt) return MLS_EINVAL;
  if (check_options(opt) != MLS_OK) return fail(ctx, MLS_EINVAL, "invalid options");
  const bool realloc = opt->precision != ctx->opt.precision || opt->stream != ctx->opt.stream;
  if (realloc && ctx->n > 0)
    return fail(ctx, MLS_EINVAL, "precision and stream are fixed once a mesh is uploaded");
  ctx->opt = *opt;
  ctx->stream = (cudaStream_t)opt->stream;
  ctx->coarse_ready = false;
  ctx->galerkin_ready = false;
  ctx->omega_eff = opt->omega > 0.0 ? opt->omega : 0.5;
  return MLS_OK;
}

mls_status mls_smoother_omega(mls_ctx* ctx, double* omega, double* lambda_max) {
  if (!ctx || !omega) return MLS_EINVAL;
  *omega = ctx->omega_eff;
  if (lambda_max) *lambda_max = ctx->omega_lmax;
  return MLS_OK;
}

double mls_tridiag_max_eig(const double* d, const double* e, int k) {
  if (!d || k < 1 || (k > 1 && !e)) return std::nan("");
  return tridiag_max_eig(d, e, k);
}

mls_status mls_set_forces(mls_ctx* ctx, const double* gravity, int contact, const double* plane_n,
                          double plane_o, double dhat, double kappa) {
  if (!ctx) return MLS_EINVAL;
  if (gravity) for (int k = 0; k < 3; ++k) ctx->grav[k] = gravity[k];
  ctx->contact = contact ? 1 : 0;
  if (contact) {
    if (!plane_n || !(dhat > 0) || !(kappa > 0)) return fail(ctx, MLS_EINVAL, "contact needs a plane, dhat > 0, kappa > 0");
    const double nn = std::sqrt(plane_n[0] * plane_n[0] + plane_n[1] * plane_n[1] + plane_n[2] * plane_n[2]);
    if (!(nn > 0)) return fail(ctx, MLS_EINVAL, "plane normal must be non-zero");
    for (int k = 0; k < 3; ++k) ctx->pn[k] = plane_n[k] / nn;
    ctx->po = plane_o / nn;
    ctx->dhat = dhat;
    ctx->kappa = kappa;
  }
  return MLS_OK;
}

mls_status mls_upload_mesh(mls_ctx* ctx, int32_t n, const double* X, int32_t t, const int32_t* tets,
                           const double* youngs, const double* poisson, const double* density,
                           const uint8_t* dirichlet) {
  if (!ctx) return MLS_EINVAL;
  if (n < 1 || t < 1 || !X || !tets || !youngs || !poisson || !density)
    return fail(ctx, MLS_EINVAL, "upload_mesh: empty mesh or null array");
  if ((int64_t)t * 16 > INT32_MAX / 2) return fail(ctx, MLS_EINVAL, "upload_mesh: too many tets");
  for (int64_t k = 0; k < 4 * (int64_t)t; ++k)
    if (tets[k] < 0 || tets[k] >= n) return fail(ctx, MLS_EINVAL, "upload_mesh: tet index out of range");
  for (int e = 0; e < t; ++e) {
    if (!(youngs[e] > 0) || !(poisson[e] > -1.0 && poisson[e] < 0.5) || !(density[e] > 0))
      return fail(ctx, MLS_EINVAL, "upload_mesh: invalid material at tet " + std::to_string(e));
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (tets[4 * e + a] == tets[4 * e + b]) return fail(ctx, MLS_EINVAL, "upload_mesh: repeated vertex in a tet");
  }
  free_all(ctx);
  ctx->n = n;
  ctx->t = t;
  // rest shapes, materials, lumped masses
  std::vector<double> h_Dminv(9 * (size_t)t), h_vol(t), h_mu(t), h_lam(t), h_mass(n, 0.0);
  for (int e = 0; e < t; ++e) {
    const double* p0 = X + 3 * (size_t)tets[4 * e];
    double D[3][3];
    for (int k = 0; k < 3; ++k) {
      const double* pk = X + 3 * (size_t)tets[4 * e + k + 1];
      for (int a = 0; a < 3; ++a) D[a][k] = pk[a] - p0[a];
    }
    const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) -
                       D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                       D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    if (!(det > 0)) return fail(ctx, MLS_EINVAL, "upload_mesh: tet " + std::to_string(e) + " has non-positive rest volume");
    const double inv[3][3] = {
        {(D[1][1] * D[2][2] - D[1][2] * D[2][1]) / det, (D[0][2] * D[2][1] - D[0][1] * D[2][2]) / det,
         (D[0][1] * D[1][2] - D[0][2] * D[1][1]) / det},
        {(D[1][2] * D[2][0] - D[1][0] * D[2][2]) / det, (D[0][0] * D[2][2] - D[0][2] * D[2][0]) / det,
         (D[0][2] * D[1][0] - D[0][0] * D[1][2]) / det},
        {(D[1][0] * D[2][1] - D[1][1] * D[2][0]) / det, (D[0][1] * D[2][0] - D[0][0] * D[2][1]) / det,
         (D[0][0] * D[1][1] - D[0][1] * D[1][0]) / det}};
    for (int k = 0; k < 3; ++k)
      for (int b = 0; b < 3; ++b) h_Dminv[(3 * k + b) * (size_t)t + e] = inv[k][b];
    h_vol[e] = det / 6.0;
    const double E = youngs[e], nu = poisson[e];
    h_mu[e] = E / (2.0 * (1.0 + nu));
    h_lam[e] = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
    for (int a = 0; a < 4; ++a) h_mass[tets[4 * e + a]] += density[e] * h_vol[e] / 4.0;
  }
  std::vector<int> vt_ptr(n + 1, 0), vt_code(4 * (size_t)t);
  for (int e = 0; e < t; ++e)
    for (int a = 0; a < 4; ++a) vt_ptr[tets[4 * e + a] + 1]++;
  for (int v = 0; v < n; ++v) vt_ptr[v + 1] += vt_ptr[v];
  {
    std::vector<int> fill(vt_ptr.begin(), vt_ptr.end() - 1);
    for (int e = 0; e < t; ++e)
      for (int a = 0; a < 4; ++a) vt_code[fill[tets[4 * e + a]]++] = 4 * e + a;
  }
  std::vector<int> tets_soa(4 * (size_t)t);
  for (int e = 0; e < t; ++e)
    for (int a = 0; a < 4; ++a) tets_soa[a * (size_t)t + e] = tets[4 * e + a];
  std::vector<Vec4d> Xp(n);
  for (int v = 0; v < n; ++v) Xp[v] = Vec4d{X[3 * v], X[3 * v + 1], X[3 * v + 2], 0.0};
  std::vector<uint8_t> pin(n, 0);
  if (dirichlet)
    for (int v = 0; v < n; ++v) pin[v] = dirichlet[v] ? 1 : 0;

  auto up = [&](void** dst, const void* src, size_t bytes) -> mls_status {
    mls_status st = dalloc(ctx, dst, bytes);
    if (st != MLS_OK) return st;
    return cuda_check(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "mesh upload");
  };
  mls_status st;
  if ((st = up((void**)&ctx->tets, tets_soa.data(), sizeof(int) * 4 * (size_t)t)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->Dminv, h_Dminv.data(), sizeof(double) * 9 * (size_t)t)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->vol, h_vol.data(), sizeof(double) * t)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->mu, h_mu.data(), sizeof(double) * t)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->lam, h_lam.data(), sizeof(double) * t)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->mass, h_mass.data(), sizeof(double) * n)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->pinned, pin.data(), n)) != MLS_OK) return st;
  ctx->h_pinned = pin;
  if ((st = up((void**)&ctx->X, Xp.data(), sizeof(Vec4d) * n)) != MLS_OK) return st;
  if ((st = up((void**)&ctx->vt_ptr, vt_ptr.data(), sizeof(int) * (n + 1))) != MLS_OK) return st;
  if ((st = up((void**)&ctx->vt_code, vt_code.data(), sizeof(int) * 4 * (size_t)t)) != MLS_OK) return st;
  ctx->mass_min = *std::min_element(h_mass.begin(), h_mass.end());
  ctx->h_mass = h_mass;
  ctx->h_X.assign(X, X + 3 * (size_t)n);
  ctx->h_tets.assign(tets, tets + 4 * (size_t)t);
  if ((st = build_pattern(ctx, nullptr)) != MLS_OK) return st;
  return alloc_state(ctx);
}

}  // extern "C"

namespace mls {
// number of eigenvalues of the symmetric tridiagonal (d, e) below x: the
// negative pivots of the LDL^T factorisation of T - x I (Sturm sequence)
static int sturm_below(const double* d, const double* e, int k, double x) {
  int count = 0;
  double q = 1.0;
  for (int i = 0; i < k; ++i) {
    q = (d[i] - x) - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
    if (q == 0.0) q = -1e-300;
    if (q < 0.0) ++count;
  }
  return count;
}

double tridiag_max_eig(const double* d, const double* e, int k) {
  double lo = INFINITY, hi = -INFINITY;  // Gershgorin interval
  for (int i = 0; i < k; ++i) {
    const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
    lo = std::min(lo, d[i] - r);
    hi = std::max(hi, d[i] + r);
  }
  // largest eigenvalue: the infimum of {x : all k eigenvalues lie below x}
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (!(mid > lo && mid < hi)) break;
    if (sturm_below(d, e, k, mid) == k) hi = mid;
    else lo = mid;
  }
  return hi;
}

static mls_status alloc_state(mls_ctx* ctx) {
  const int n = ctx->n, t = ctx->t;
  mls_status st;
  const size_t v4 = sizeof(Vec4d) * (size_t)n;
  Vec4d** v4bufs[] = {&ctx->xk, &ctx->xt, &ctx->xtil, &ctx->dir, &ctx->grad, &ctx->tmp4};
  for (Vec4d** b : v4bufs)
    if ((st = dalloc(ctx, (void**)b, v4)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->egrad, sizeof(double) * 12 * (size_t)t)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->stage, sizeof(double) * 9 * (size_t)n)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->ehess, (size_t)element_bytes(ctx) * 78 * t)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->hval, (size_t)storage_bytes(ctx) * 288 * ctx->n_groups)) != MLS_OK) return st;
  const int vb = solve_bytes(ctx);
  if ((st = dalloc(ctx, &ctx->dinv, (size_t)vb * 9 * n)) != MLS_OK) return st;
  void** sv[] = {&ctx->vb, &ctx->vx, &ctx->vr, &ctx->vz, &ctx->vp, &ctx->vq, &ctx->vw, &ctx->vz2};
  for (void** b : sv)
    if ((st = dalloc(ctx, b, (size_t)vb * 4 * n)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->pcg, sizeof(PcgScalars))) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->lz, sizeof(double) * (2 * kLanczosSteps + 1))) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->pcg_fix, sizeof(unsigned long long) * kFixWords)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemset(ctx->pcg_fix, 0, sizeof(unsigned long long) * kFixWords), "sum init")) != MLS_OK)
    return st;
  if ((st = dalloc(ctx, (void**)&ctx->persist_part, sizeof(double) * 4 * kMaxPersistBlocks)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->persist_bar, 64)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemset(ctx->persist_bar, 0, 64), "barrier init")) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->dscal, sizeof(double) * 16)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->red.partials, sizeof(double) * 4 * kMaxPartials)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&ctx->red.counter, sizeof(unsigned) * RS_COUNT)) != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemset(ctx->red.counter, 0, sizeof(unsigned) * RS_COUNT), "counter init");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemset(ctx->tmp4, 0, v4), "zero init");
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaMemset(ctx->hval, 0, (size_t)storage_bytes(ctx) * 288 * ctx->n_groups), "H init");
}

// ---- the timestep -------------------------------------------------------------------------
static const double kArmijo = 1e-4;
static const double kRoundingRegime = 1e-13;
static const int kMaxHalvings = 60;

static mls_status assemble_at(mls_ctx* ctx, const Vec4d* x, double* gnorm) {
  mls_status st;
  int tk = prof_begin(ctx, MLS_PROF_ELEMENTS);
  if ((st = launch_eval_elements(ctx, x, nullptr)) != MLS_OK) return st;
  prof_end(ctx, tk);
  tk = prof_begin(ctx, MLS_PROF_ASSEMBLE);
  // mesh-mesh pairs first: their gradient enters the gather, their blocks H
  if ((st = contact_assemble(ctx, x)) != MLS_OK) return st;
  if ((st = launch_gather_grad(ctx, x, ctx->dscal + 2)) != MLS_OK) return st;
  if ((st = launch_assemble(ctx, x)) != MLS_OK) return st;
  if ((st = contact_merge(ctx, ctx->hval, ctx->dinv, true)) != MLS_OK) return st;
  prof_end(ctx, tk);
  ctx->assembled = true;
  if (gnorm) {
    double g2 = 0;
    if ((st = read_scalar(ctx, ctx->dscal + 2, &g2)) != MLS_OK) return st;
    *gnorm = std::sqrt(g2);
  }
  return MLS_OK;
}

// The paper's inexact direction (Alg. 1, Alg. 2): the subspace direction
// d_s = U (U^T H U)^{-1} U^T (-g) with the factored Galerkin operator (the
// affine level adds nothing to an exact solve in span U, which contains the
// affine motions), then refine_iters block-Jacobi CG iterations on
// H d_f = -g - H d_s from d_f = 0 (Sec. 3.8: a fixed count of Jacobi-
// preconditioned CG iterations).  Leaves d = d_s + d_f in vx (solve
// precision) and returns sum_v |d_s,v|_2 and the CG iterations run.
// H_lag refresh: the current element Hessians become the lagged ones
constexpr double kLagAlpha = 0.5;
constexpr int kLagMinAge = 5;
static mls_status hessian_lag_refresh(mls_ctx* ctx) {
  mls_status st;
  const size_t eb = (size_t)78 * ctx->t * (ctx->opt.precision == MLS_FP64 ? 8 : 4);
  if (!ctx->ehess_lag) {
    if ((st = dalloc(ctx, &ctx->ehess_lag, eb)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->hval_lag, (size_t)storage_bytes(ctx) * 288 * ctx->n_groups)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->dinv_lag, (size_t)solve_bytes(ctx) * 9 * ctx->n)) != MLS_OK) return st;
  }
  ctx->lag_age = 0;
  ctx->lag_nalpha = 0;
  return cuda_check(ctx, cudaMemcpyAsync(ctx->ehess_lag, ctx->ehess, eb, cudaMemcpyDeviceToDevice, ctx->stream),
                    "H_lag refresh");
}

// The subspace direction of Alg. 2 as printed (direction 2), into vw:
// the affine level (one handle at the centre of mass, phi = 1, Sec. 3.4)
// solved on its 12 x 12 operator A_a = T^T (U^T H U) T, T the coordinates of
// an affine motion in the SMS basis (the SMS weights sum to one), then the
// SMS level by block-Jacobi PCG on the residual (sms_pcg).  The affine level
// is left out on meshes with Dirichlet vertices, whose SMS weights do not
// sum to one there.
static mls_status subspace_direction_literal(mls_ctx* ctx, int* sub_iters) {
  mls_status st;
  const Basis& B = ctx->basis;
  const int m = B.m, r = 12 * m;
  const bool fp64 = ctx->opt.precision == MLS_FP64;
  const size_t vb = fp64 ? sizeof(double) : sizeof(float);
  if ((st = launch_restrict(ctx, ctx->vb, ctx->cvec)) != MLS_OK) return st;  // U^T (-g)
  bool affine = true;
  for (int v = 0; v < ctx->n && affine; ++v) affine = !ctx->h_pinned[v];
  *sub_iters = 0;
  std::vector<double> ca(r, 0.0);
  if (affine) {
    // centre of mass and the offsets d_j = o_j - o_a
    double om[3] = {0, 0, 0}, mt = 0;
    for (int v = 0; v < ctx->n; ++v) {
      mt += ctx->h_mass[v];
      for (int c = 0; c < 3; ++c) om[c] += ctx->h_mass[v] * ctx->h_X[3 * (size_t)v + c];
    }
    for (int c = 0; c < 3; ++c) om[c] /= mt;
    std::vector<double> d(3 * (size_t)m);
    for (int j = 0; j < m; ++j)
      for (int c = 0; c < 3; ++c) d[3 * j + c] = B.h_origins[3 * (size_t)j + c] - om[c];
    // M = A_s T on the device, then A_a = T^T M and b_a = T^T U^T(-g) here
    if ((st = affine_operator(ctx, om)) != MLS_OK) return st;
    std::vector<double> M((size_t)r * 12), cg(r);
    std::vector<float> cgf;
    if ((st = cuda_check(ctx, cudaMemcpyAsync(M.data(), ctx->sms_m, sizeof(double) * M.size(), cudaMemcpyDeviceToHost,
                                              ctx->stream), "affine operator")) != MLS_OK)
      return st;
    if (fp64) {
      st = cuda_check(ctx, cudaMemcpyAsync(cg.data(), ctx->cvec, sizeof(double) * r, cudaMemcpyDeviceToHost, ctx->stream),
                      "U^T g");
    } else {
      cgf.resize(r);
      st = cuda_check(ctx, cudaMemcpyAsync(cgf.data(), ctx->cvec, sizeof(float) * r, cudaMemcpyDeviceToHost, ctx->stream),
                      "U^T g");
    }
    if (st != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "affine sync")) != MLS_OK) return st;
    if (!fp64)
      for (int i = 0; i < r; ++i) cg[i] = cgf[i];
    // T^T applied to a coarse vector y (length r) and to the columns of M:
    // (T^T y)[(c, 0)] = sum_j y[12j+4c]; (T^T y)[(c, l)] = sum_j y[12j+4c+l] + d_{j,l} y[12j+4c]
    auto tt = [&](auto get, double out[12]) {
      for (int k = 0; k < 12; ++k) out[k] = 0.0;
      for (int j = 0; j < m; ++j)
        for (int c = 0; c < 3; ++c) {
          const double y0 = get(12 * j + 4 * c);
          out[4 * c] += y0;
          for (int l = 1; l < 4; ++l) out[4 * c + l] += get(12 * j + 4 * c + l) + d[3 * j + l - 1] * y0;
        }
    };
    double Aa[12][12], ba[12];
    for (int col = 0; col < 12; ++col) {
      double out[12];
      tt([&](int i) { return M[(size_t)i * 12 + col]; }, out);
      for (int k = 0; k < 12; ++k) Aa[k][col] = out[k];
    }
    tt([&](int i) { return cg[i]; }, ba);
    // 12 x 12 Cholesky solve of A_a q_a = b_a (the block-Jacobi PCG of a
    // single 12 x 12 block converges in one step)
    double L[12][12] = {};
    for (int i = 0; i < 12; ++i)
      for (int j = 0; j <= i; ++j) {
        double sum = 0.5 * (Aa[i][j] + Aa[j][i]);
        for (int k = 0; k < j; ++k) sum -= L[i][k] * L[j][k];
        if (i == j) {
          if (!(sum > 0.0)) return fail(ctx, MLS_ECHOL, "affine level: operator not positive definite");
          L[i][i] = std::sqrt(sum);
        } else {
          L[i][j] = sum / L[j][j];
        }
      }
    double y[12], qa[12];
    for (int i = 0; i < 12; ++i) {
      double sum = ba[i];
      for (int k = 0; k < i; ++k) sum -= L[i][k] * y[k];
      y[i] = sum / L[i][i];
    }
    for (int i = 11; i >= 0; --i) {
      double sum = y[i];
      for (int k = i + 1; k < 12; ++k) sum -= L[k][i] * qa[k];
      qa[i] = sum / L[i][i];
    }
    // c_a = T q_a
    for (int j = 0; j < m; ++j)
      for (int c = 0; c < 3; ++c) {
        double t0 = qa[4 * c];
        for (int l = 1; l < 4; ++l) {
          t0 += d[3 * j + l - 1] * qa[4 * c + l];
          ca[12 * j + 4 * c + l] = qa[4 * c + l];
        }
        ca[12 * j + 4 * c] = t0;
      }
    *sub_iters += 1;
    // d_a = U c_a into vw; right-hand side of the SMS level U^T (-g - H d_a)
    if (fp64) {
      st = cuda_check(ctx, cudaMemcpyAsync(ctx->cvec2, ca.data(), vb * r, cudaMemcpyHostToDevice, ctx->stream), "c_a");
    } else {
      cgf.assign(ca.begin(), ca.end());
      st = cuda_check(ctx, cudaMemcpyAsync(ctx->cvec2, cgf.data(), vb * r, cudaMemcpyHostToDevice, ctx->stream), "c_a");
    }
    if (st != MLS_OK) return st;
    if ((st = launch_prolong(ctx, ctx->cvec2, ctx->vw, false)) != MLS_OK) return st;
    if ((st = launch_residual(ctx, ctx->vb, ctx->vw, ctx->vz2, nullptr)) != MLS_OK) return st;
    if ((st = launch_restrict(ctx, ctx->vz2, ctx->cvec)) != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "affine upload")) != MLS_OK) return st;
  } else {
    if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->vw, 0, (size_t)ctx->n * 4 * vb, ctx->stream), "d_a = 0")) != MLS_OK)
      return st;
  }
  int it = 0;
  if ((st = sms_pcg(ctx, ctx->cvec, ctx->opt.sub_rtol, 100000, &it)) != MLS_OK) return st;
  *sub_iters += it;
  return launch_prolong(ctx, ctx->cvec, ctx->vw, true);  // d_s = d_a + U q
}

static mls_status paper_direction(mls_ctx* ctx, double* ds_norm, int* cg_iters, int* sub_iters) {
  mls_status st;
  *sub_iters = 0;
  if (ctx->opt.direction == 2) {
    if ((st = subspace_direction_literal(ctx, sub_iters)) != MLS_OK) return st;
  } else {
    if ((st = launch_restrict(ctx, ctx->vb, ctx->cvec)) != MLS_OK) return st;
    if ((st = coarse_apply(ctx, ctx->cvec, ctx->cvec2)) != MLS_OK) return st;
    if ((st = launch_prolong(ctx, ctx->cvec2, ctx->vw, false)) != MLS_OK) return st;
  }
  if ((st = launch_from_solve(ctx, ctx->vw, ctx->dir)) != MLS_OK) return st;
  if ((st = vnorm_sum(ctx, ctx->dir, ds_norm)) != MLS_OK) return st;
  // right-hand side of the refinement: vb = -g - H d_s (through vz2)
  const size_t vbytes = (size_t)ctx->n * (ctx->opt.precision == MLS_FP64 ? sizeof(Vec4d) : sizeof(Vec4f));
  if ((st = launch_residual(ctx, ctx->vb, ctx->vw, ctx->vz2, nullptr)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->vb, ctx->vz2, vbytes, cudaMemcpyDeviceToDevice, ctx->stream),
                       "refinement rhs")) != MLS_OK)
    return st;
  const int pc = ctx->opt.preconditioner;
  ctx->opt.preconditioner = MLS_PRECOND_BLOCK_JACOBI;
  const bool lag = ctx->opt.hessian_lag && ctx->hval_lag;
  if (lag) {  // the refinement solves H_lag d_f = r (Sec. 3.7.2)
    std::swap(ctx->hval, ctx->hval_lag);
    std::swap(ctx->dinv, ctx->dinv_lag);
  }
  double rel = 0;
  *cg_iters = 0;
  if (ctx->opt.refine_iters > 0) {
    st = pcg_solve(ctx, 0.0, ctx->opt.refine_iters, cg_iters, &rel);
  } else {
    st = cuda_check(ctx, cudaMemsetAsync(ctx->vx, 0, vbytes, ctx->stream), "zero d_f");
  }
  if (lag) {
    std::swap(ctx->hval, ctx->hval_lag);
    std::swap(ctx->dinv, ctx->dinv_lag);
  }
  ctx->opt.preconditioner = pc;
  if (st != MLS_OK && st != MLS_ENOTCONV) return st;
  return launch_add_solve(ctx, ctx->vx, ctx->vw);
}

// a lagged coarse factor is stale when the first PCG solve of a step takes
// more than kLagStaleRatio x (iterations after the last build) + kLagStaleSlack
constexpr double kLagStaleRatio = 1.5;
constexpr int kLagStaleSlack = 8;

static mls_status newton_loop(mls_ctx* ctx, mls_stats* stats) {
  mls_stats S{};
  mls_status st;
  const int64_t shifts0 = ctx->coarse_shift_count;
  if (ctx->coarse_ready) ctx->coarse_age_steps++;
  const double h = ctx->h_step;  // the timestep (ctx->h is the potential's step, 2h/3 for BDF2)
  const double gmag = std::sqrt(ctx->grav[0] * ctx->grav[0] + ctx->grav[1] * ctx->grav[1] + ctx->grav[2] * ctx->grav[2]);
  const double scale0 = h * h * std::max(gmag, 1e-30);
  double E = 0;
  int infeasible = 0;
  // friction between bodies: its pairs and frames, lagged at x^t for the step
  if ((st = contact_friction_lag(ctx)) != MLS_OK) return st;
  // x^t must be feasible; start from x_tilde when it is, else from x^t
  if ((st = launch_energy(ctx, ctx->xt, ctx->tmp4, 0.0, &E, &infeasible)) != MLS_OK) return st;
  if (infeasible) return fail(ctx, MLS_EINVERTED, "x^t has an inverted tet or a vertex on/below the plane");
  if (!std::isfinite(E)) return fail(ctx, MLS_ENONFINITE, "non-finite energy at x^t");
  if (ctx->cs.on) {
    // with bodies the straight path x^t -> x_tilde is cut by the CCD filter
    // first (a straight move could pass one body through another)
    if ((st = launch_diff_state(ctx, ctx->xk, ctx->xt, ctx->dir)) != MLS_OK) return st;
    double a0 = 1.0;
    if ((st = launch_ccd(ctx, ctx->xt, ctx->dir, &a0)) != MLS_OK) return st;
    if ((st = launch_xpay_state(ctx, ctx->xt, ctx->dir, a0, ctx->xk)) != MLS_OK) return st;
  }
  if ((st = launch_energy(ctx, ctx->xk, ctx->tmp4, 0.0, &E, &infeasible)) != MLS_OK) return st;
  if (infeasible || !std::isfinite(E)) {
    st = cuda_check(ctx, cudaMemcpyAsync(ctx->xk, ctx->xt, sizeof(Vec4d) * ctx->n, cudaMemcpyDeviceToDevice,
                                         ctx->stream), "restart from x^t");
    if (st != MLS_OK) return st;
    contact_invalidate(ctx);
  }
  const bool two_level = ctx->opt.preconditioner == MLS_PRECOND_TWO_LEVEL;
  if (two_level && !ctx->has_basis) return fail(ctx, MLS_EINVAL, "two-level preconditioner needs mls_upload_basis");
  const bool paper = ctx->opt.direction >= 1;
  if (paper && !two_level) return fail(ctx, MLS_EINVAL, "the paper's direction needs the two-level preconditioner");
  {
    int used = 0;
    if ((st = warm_start_begin(ctx, &used)) != MLS_OK) return st;
    S.warm_start_used = used;
  }
  const double eta_floor = ctx->opt.precision == MLS_FP64 ? 1e-13 : 1e-6;
  double g0 = -1.0;
  mls_status result = MLS_ENOTCONV;
  for (int it = 0; it < ctx->opt.max_newton; ++it) {
    double gnorm = 0;
    if ((st = assemble_at(ctx, ctx->xk, &gnorm)) != MLS_OK) return st;
    if (!std::isfinite(gnorm)) return fail(ctx, MLS_ENONFINITE, "non-finite gradient");
    if (g0 < 0) g0 = gnorm;
    S.grad_norm = gnorm;
    S.newton_iters = it + 1;
    if (gnorm == 0.0) { S.step_rel = 0.0; result = MLS_OK; break; }
    bool lagged_first = false;
    if (two_level) {
      const int k = ctx->opt.coarse_refresh;
      const bool ready = ctx->opt.direction == 2 ? ctx->galerkin_ready : ctx->coarse_ready;
      bool rebuild = k == 0 || it % k == 0 || !ready || ctx->coarse_stale;
      // a lagged factor only preconditions: the paper's direction solves with it
      if (it == 0 && !paper && ctx->coarse_ready && !ctx->coarse_stale &&
          ctx->coarse_age_steps <= ctx->opt.coarse_lag_steps)
        rebuild = false;
      if (rebuild) {
        // the literal subspace solve needs U^T H U itself, not a factor
        st = ctx->opt.direction == 2 ? build_coarse_unfactored(ctx) : build_coarse(ctx);
        // a coarse operator that stays indefinite after the shift retries:
        // this Newton iteration preconditions with block Jacobi, and the
        // next one tries the coarse build again at its own iterate
        if (st == MLS_ECHOL && !paper) {
          ctx->coarse_fallback = true;
          S.coarse_fallbacks++;
        } else if (st != MLS_OK) {
          return st;
        } else {
          ctx->coarse_fallback = false;
          S.coarse_builds++;
        }
      }
      lagged_first = it == 0 && !rebuild;
    }
    if (it == 0 && (st = warm_start_first_iteration(ctx)) != MLS_OK) return st;
    if (paper) {
      if (ctx->opt.hessian_lag) {
        // H_lag (Sec. 3.7.2): refreshed at the step's first iteration and when
        // the mean of the last three step sizes falls below kLagAlpha, at most
        // once every kLagMinAge iterations; contact and friction blocks fresh
        double ma = 0.0;
        const int na = std::min(ctx->lag_nalpha, 3);
        for (int k = 0; k < na; ++k) ma += ctx->lag_alpha[k];
        ma = na ? ma / na : 1.0;
        if (it == 0 || (na == 3 && ma < kLagAlpha && ctx->lag_age >= kLagMinAge)) {
          if ((st = hessian_lag_refresh(ctx)) != MLS_OK) return st;
          S.hessian_refreshes++;
        }
        if ((st = launch_assemble_lagged(ctx, ctx->xk)) != MLS_OK) return st;
        ctx->lag_age++;
      }
      double ds_norm = 0;
      int cg = 0, sub = 0;
      if ((st = paper_direction(ctx, &ds_norm, &cg, &sub)) != MLS_OK) return st;
      S.pcg_iters += cg;
      S.subspace_iters += sub;
      if ((st = launch_from_solve(ctx, ctx->vx, ctx->dir)) != MLS_OK) return st;
      double gd = 0;
      if ((st = dot4(ctx, ctx->grad, ctx->dir, &gd)) != MLS_OK) return st;
      if (!std::isfinite(gd)) return fail(ctx, MLS_ENONFINITE, "non-finite Newton direction");
      if (!(gd < 0)) return fail(ctx, MLS_ELINESEARCH, "Newton direction is not a descent direction");
      double alpha = 1.0;
      if ((st = launch_ccd(ctx, ctx->xk, ctx->dir, &alpha)) != MLS_OK) return st;
      double E0 = 0;
      if ((st = launch_energy(ctx, ctx->xk, ctx->dir, 0.0, &E0, &infeasible)) != MLS_OK) return st;
      bool accepted = false;
      for (int hv = 0; hv <= kMaxHalvings; ++hv) {
        if ((st = launch_energy(ctx, ctx->xk, ctx->dir, alpha, &E, &infeasible)) != MLS_OK) return st;
        S.line_search_trials++;
        if (!infeasible && (std::fabs(kArmijo * alpha * gd) <= kRoundingRegime * std::fabs(E0) ||
                            E <= E0 + kArmijo * alpha * gd)) {
          accepted = true;
          break;
        }
        alpha *= 0.5;
      }
      if (!accepted) return fail(ctx, MLS_ELINESEARCH, "line search found no acceptable step");
      if ((st = launch_axpy_state(ctx, ctx->xk, ctx->dir, alpha)) != MLS_OK) return st;
      ctx->lag_alpha[ctx->lag_nalpha % 3] = alpha;
      ctx->lag_nalpha++;
      S.step_rel = ds_norm / (h * ctx->n);
      if (S.step_rel < ctx->opt.paper_tol) { result = MLS_OK; break; }
      continue;
    }
    double eta = std::min(ctx->opt.pcg_rtol, std::sqrt(gnorm / g0));
    eta = std::max(eta, eta_floor);
    // absolute floor: H >= M, so |d - d*|_2 <= |r|_2 / m_min; a residual below
    // 0.01 newton_tol x scale x m_min cannot move the step test
    double xdisp0 = 0, dn0 = 0;
    if ((st = launch_norms(ctx, ctx->tmp4, &dn0, &xdisp0)) != MLS_OK) return st;
    const double abs_floor = 0.01 * ctx->opt.newton_tol * std::max(xdisp0, scale0) * ctx->mass_min;
    eta = std::max(eta, abs_floor / gnorm);
    int iters = 0;
    double rel = 0;
    st = pcg_solve(ctx, eta, ctx->opt.max_pcg, &iters, &rel);
    // automatic damping: a breakdown means omega lambda_max(D^{-1} H) reached 2
    // since the estimate (taken at the last coarse build); retry with a smaller omega
    for (int retry = 0; st == MLS_ENONFINITE && two_level && ctx->opt.omega == 0.0 && retry < 3; ++retry) {
      S.pcg_iters += iters;
      ctx->omega_eff *= 0.8;
      st = pcg_solve(ctx, eta, ctx->opt.max_pcg, &iters, &rel);
    }
    S.pcg_iters += iters;
    if (st != MLS_OK && st != MLS_ENOTCONV) return st;
    // quality of a lagged coarse factor: the first solve of a step against
    // the first solve of a step after the last build; a much harder solve
    // marks the factor stale, and the next Newton iteration rebuilds it
    if (it == 0 && two_level) {
      if (ctx->coarse_ref_pending) {
        ctx->coarse_ref_iters = iters;
        ctx->coarse_ref_pending = false;
      } else if (lagged_first && iters > kLagStaleRatio * ctx->coarse_ref_iters + kLagStaleSlack) {
        ctx->coarse_stale = true;
      }
    }
    if ((st = launch_from_solve(ctx, ctx->vx, ctx->dir)) != MLS_OK) return st;
    double dinf = 0, xdisp = 0;
    if ((st = launch_norms(ctx, ctx->dir, &dinf, &xdisp)) != MLS_OK) return st;
    if (!std::isfinite(dinf)) return fail(ctx, MLS_ENONFINITE, "non-finite Newton direction");
    const double step_rel = dinf / std::max(xdisp, scale0);
    S.step_rel = step_rel;
    double gd = 0;
    if ((st = dot4(ctx, ctx->grad, ctx->dir, &gd)) != MLS_OK) return st;
    if (step_rel <= ctx->opt.newton_tol) {
      // converged: apply the final (tiny) direction in full when feasible
      // and, with bodies, when the mesh-mesh CCD filter does not cut it (a
      // feasible end point does not rule out a vertex that passed through a
      // triangle on the way)
      if ((st = launch_energy(ctx, ctx->xk, ctx->dir, 1.0, &E, &infeasible)) != MLS_OK) return st;
      S.line_search_trials++;
      if (!infeasible && ctx->cs.on) {
        double t = 1.0;
        if ((st = contact_ccd(ctx, ctx->xk, ctx->dir, &t)) != MLS_OK) return st;
        infeasible = t < 1.0;
      }
      if (!infeasible) {
        if ((st = launch_axpy_state(ctx, ctx->xk, ctx->dir, 1.0)) != MLS_OK) return st;
      }
      result = MLS_OK;
      break;
    }
    if (!(gd < 0)) return fail(ctx, MLS_ELINESEARCH, "Newton direction is not a descent direction");
    double alpha = 1.0;
    if ((st = launch_ccd(ctx, ctx->xk, ctx->dir, &alpha)) != MLS_OK) return st;
    double E0 = 0;
    if ((st = launch_energy(ctx, ctx->xk, ctx->dir, 0.0, &E0, &infeasible)) != MLS_OK) return st;
    bool accepted = false;
    for (int hv = 0; hv <= kMaxHalvings; ++hv) {
      if ((st = launch_energy(ctx, ctx->xk, ctx->dir, alpha, &E, &infeasible)) != MLS_OK) return st;
      S.line_search_trials++;
      if (!infeasible) {
        if (std::fabs(kArmijo * alpha * gd) <= kRoundingRegime * std::fabs(E0) ||
            E <= E0 + kArmijo * alpha * gd) {
          accepted = true;
          break;
        }
      }
      alpha *= 0.5;
    }
    if (!accepted) return fail(ctx, MLS_ELINESEARCH, "line search found no acceptable step");
    if ((st = launch_axpy_state(ctx, ctx->xk, ctx->dir, alpha)) != MLS_OK) return st;
  }
  if ((st = launch_energy(ctx, ctx->xk, ctx->tmp4, 0.0, &E, &infeasible)) != MLS_OK) return st;
  if (result == MLS_OK && (st = warm_start_end(ctx)) != MLS_OK) return st;
  prof_flush(ctx);
  S.energy = E;
  S.coarse_shifts = (int)(ctx->coarse_shift_count - shifts0);
  S.contact_pairs = ctx->cs.npt + ctx->cs.nee;
  if (stats) *stats = S;
  if (result != MLS_OK) return fail(ctx, result, "Newton reached its iteration cap");
  return MLS_OK;
}

// The block-Jacobi fallback of a failed coarse build lasts one Newton loop
static mls_status newton(mls_ctx* ctx, mls_stats* stats) {
  ctx->coarse_fallback = false;
  const mls_status st = newton_loop(ctx, stats);
  ctx->coarse_fallback = false;
  return st;
}

static mls_status check_mesh(mls_ctx* ctx) {
  if (!ctx) return MLS_EINVAL;
  if (ctx->n < 1) return fail(ctx, MLS_EINVAL, "no mesh uploaded");
  return MLS_OK;
}

// Stage calls set up the timestep state from (x_t, v_t, dt) without running Newton
static mls_status set_timestep(mls_ctx* ctx, const double* x_t, const double* v_t, double dt) {
  if (!(dt > 0)) return fail(ctx, MLS_EINVAL, "dt must be positive");
  ctx->h = dt;
  ctx->h_step = dt;
  return launch_predictor(ctx, x_t, v_t, dt);
}

// BDF2 (Sec. 3.1): Eq. IP with alpha = 4/9 is the implicit-Euler potential of
// the step 2 dt / 3 around the BDF2 predictor, so the Newton loop runs unchanged
static mls_status set_timestep_bdf2(mls_ctx* ctx, const double* x_t, const double* v_t, const double* x_prev,
                                    const double* v_prev, double dt) {
  if (!(dt > 0)) return fail(ctx, MLS_EINVAL, "dt must be positive");
  ctx->h = 2.0 * dt / 3.0;
  ctx->h_step = dt;
  return launch_predictor_bdf2(ctx, x_t, v_t, x_prev, v_prev, dt);
}

}  // namespace mls

extern "C" {

mls_status mls_newton_step(mls_ctx* ctx, const double* x, const double* v, double dt, double* dx_out,
                           mls_stats* stats_out) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !v || !dx_out) return fail(ctx, MLS_EINVAL, "null state pointer");
  const int64_t l0 = ctx->launches;
  if ((st = set_timestep(ctx, x, v, dt)) != MLS_OK) return st;
  mls_status res = newton(ctx, stats_out);
  if (res != MLS_OK && res != MLS_ENOTCONV) return res;
  if ((st = launch_disp_out(ctx, dx_out)) != MLS_OK) return st;
  if (stats_out) stats_out->kernel_launches = ctx->launches - l0;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "newton_step sync");
  return st != MLS_OK ? st : res;
}

mls_status mls_newton_step_bdf2(mls_ctx* ctx, const double* x, const double* v, const double* x_prev,
                                const double* v_prev, double dt, double* dx_out, mls_stats* stats_out) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !v || !x_prev || !v_prev || !dx_out) return fail(ctx, MLS_EINVAL, "null state pointer");
  const int64_t l0 = ctx->launches;
  if ((st = set_timestep_bdf2(ctx, x, v, x_prev, v_prev, dt)) != MLS_OK) return st;
  mls_status res = newton(ctx, stats_out);
  if (res != MLS_OK && res != MLS_ENOTCONV) return res;
  if ((st = launch_disp_out(ctx, dx_out)) != MLS_OK) return st;
  if (stats_out) stats_out->kernel_launches = ctx->launches - l0;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "newton_step_bdf2 sync");
  return st != MLS_OK ? st : res;
}

mls_status mls_set_friction(mls_ctx* ctx, double mu, double eps_v) {
  if (!ctx) return MLS_EINVAL;
  if (!(mu >= 0.0) || !std::isfinite(mu)) return fail(ctx, MLS_EINVAL, "friction coefficient must be >= 0");
  if (mu > 0.0 && !(eps_v > 0.0 && std::isfinite(eps_v)))
    return fail(ctx, MLS_EINVAL, "friction needs a positive mollifier velocity eps_v");
  if (mu > 0.0 && !ctx->contact && !ctx->cs.on)
    return fail(ctx, MLS_EINVAL, "friction needs the contact plane (mls_set_forces) or bodies (mls_set_bodies)");
  ctx->fric_mu = mu;
  if (mu > 0.0) ctx->fric_eps_v = eps_v;
  return MLS_OK;
}

mls_status mls_newton_step_host(mls_ctx* ctx, const double* x, const double* v, double dt, double* dx_out,
                                mls_stats* stats_out) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !v || !dx_out) return fail(ctx, MLS_EINVAL, "null state pointer");
  const size_t bytes = sizeof(double) * 3 * (size_t)ctx->n;
  double* dev = ctx->stage;
  st = cuda_check(ctx, cudaMemcpyAsync(dev, x, bytes, cudaMemcpyHostToDevice, ctx->stream), "x upload");
  if (st == MLS_OK) st = cuda_check(ctx, cudaMemcpyAsync(dev + 3 * (size_t)ctx->n, v, bytes, cudaMemcpyHostToDevice, ctx->stream), "v upload");
  mls_status res = st;
  if (st == MLS_OK) res = mls_newton_step(ctx, dev, dev + 3 * (size_t)ctx->n, dt, dev + 6 * (size_t)ctx->n, stats_out);
  if (res == MLS_OK || res == MLS_ENOTCONV) {
    st = cuda_check(ctx, cudaMemcpyAsync(dx_out, dev + 6 * (size_t)ctx->n, bytes, cudaMemcpyDeviceToHost, ctx->stream), "dx download");
    if (st == MLS_OK) st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "host step sync");
    if (st != MLS_OK) res = st;
  }
  cudaStreamSynchronize(ctx->stream);
  return res;
}

mls_status mls_upload_basis(mls_ctx* ctx, int32_t m, const double* origins, const int32_t* vrow,
                            const int32_t* handle, const double* phi) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!origins || !vrow || (!handle && vrow[ctx->n] > 0) || (!phi && vrow[ctx->n] > 0))
    return fail(ctx, MLS_EINVAL, "upload_basis: null array");
  if (ctx->has_basis) {
    Basis& B = ctx->basis;
    void* old[] = {B.vrow, B.vh, B.vphi, B.hrow, B.hv, B.hphi, B.origins, B.yrow, B.yh, B.yslot, B.hn_row, B.hn,
                   B.ent_ptr, B.ent_y, B.ent_v, B.ent_phi, B.ypair_row, B.chunk_ptr, B.chunk_beg, B.slot_row,
                   B.vcoef, B.hcoef, B.rchunk_handle, B.rchunk_beg, B.rchunk_ptr, B.rpart, B.rcount,
                   ctx->gpart, ctx->yval, ctx->Ac, ctx->Acopy,
                   ctx->Linv, ctx->LinvT, ctx->Ainv, ctx->cvec, ctx->cvec2, ctx->chol_info, ctx->chol_tinv,
                   ctx->oz_fwd, ctx->oz_e, ctx->sms_buf, ctx->sms_cg, ctx->sms_m,
                   ctx->Am, ctx->Wm, ctx->WmT, ctx->ws_c, ctx->ws_c2, ctx->ws_tmp, ctx->ws_hist, ctx->ws_qg,
                   ctx->ws_qtilde, ctx->ws_qnext, ctx->ws_feat, ctx->ws_target, ctx->ws_pred, ctx->ws_hsave};
    for (void* p : old) dfree(ctx, p);
    ctx->Am = nullptr; ctx->Wm = ctx->WmT = ctx->ws_c = ctx->ws_c2 = ctx->ws_tmp = nullptr;
    ctx->ws_hist = ctx->ws_qg = ctx->ws_qtilde = ctx->ws_qnext = nullptr;
    ctx->ws_feat = ctx->ws_target = ctx->ws_pred = nullptr;
    ctx->ws_hsave = nullptr;
    ctx->oz_fwd = nullptr;
    ctx->oz_e = nullptr;
    ctx->sms_buf = nullptr;
    ctx->sms_cg = nullptr;
    ctx->sms_m = nullptr;
    ctx->ws_ready = ctx->ws_enabled = ctx->ws_hist_valid = ctx->ws_record = false;
    ctx->ws_mlp = nullptr;
    ctx->basis = Basis{};
    ctx->has_basis = false;
    ctx->coarse_ready = false;
    ctx->galerkin_ready = false;
  }
  return basis_upload(ctx, m, origins, vrow, handle, phi);
}

mls_status mls_upload_cubature(mls_ctx* ctx, const double* scale) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (ctx->cub_scale) dfree(ctx, ctx->cub_scale);
  if (ctx->hval_cub) dfree(ctx, ctx->hval_cub);
  ctx->cub_scale = nullptr;
  ctx->hval_cub = nullptr;
  ctx->coarse_ready = false;
  ctx->galerkin_ready = false;
  if (!scale) return MLS_OK;
  for (int e = 0; e < ctx->t; ++e)
    if (!(scale[e] >= 0.0) || !std::isfinite(scale[e])) return fail(ctx, MLS_EINVAL, "cubature scale must be finite and >= 0");
  if ((st = dalloc(ctx, (void**)&ctx->cub_scale, sizeof(double) * (size_t)ctx->t)) != MLS_OK) return st;
  if ((st = dalloc(ctx, &ctx->hval_cub, (size_t)storage_bytes(ctx) * 288 * ctx->n_groups)) != MLS_OK) return st;
  return cuda_check(ctx, cudaMemcpy(ctx->cub_scale, scale, sizeof(double) * (size_t)ctx->t, cudaMemcpyHostToDevice),
                    "cubature upload");
}

mls_status mls_eval_elements(mls_ctx* ctx, const double* x, double* energy, double* grad, double* hess) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x) return fail(ctx, MLS_EINVAL, "null x");
  if ((st = launch_pack(ctx, x, ctx->tmp4)) != MLS_OK) return st;
  if ((st = launch_eval_elements(ctx, ctx->tmp4, energy)) != MLS_OK) return st;
  if (grad) {
    // [12][t] SoA -> [t][12]
    std::vector<double> h(12 * (size_t)ctx->t), o(12 * (size_t)ctx->t);
    st = cuda_check(ctx, cudaMemcpyAsync(h.data(), ctx->egrad, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream), "grad readback");
    if (st != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "grad sync")) != MLS_OK) return st;
    for (int e = 0; e < ctx->t; ++e)
      for (int k = 0; k < 12; ++k) o[12 * (size_t)e + k] = h[(size_t)k * ctx->t + e];
    st = cuda_check(ctx, cudaMemcpyAsync(grad, o.data(), sizeof(double) * o.size(), cudaMemcpyHostToDevice, ctx->stream), "grad out");
    if (st != MLS_OK) return st;
  }
  if (hess) {
    if ((st = launch_expand_hessian(ctx, hess)) != MLS_OK) return st;
  }
  // restore zero scratch
  st = cuda_check(ctx, cudaMemsetAsync(ctx->tmp4, 0, sizeof(Vec4d) * ctx->n, ctx->stream), "scratch reset");
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "eval sync");
}

mls_status mls_assemble(mls_ctx* ctx, const double* x, const double* x_t, const double* v_t, double dt,
                        double* grad_out) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !x_t || !v_t) return fail(ctx, MLS_EINVAL, "null pointer");
  if ((st = set_timestep(ctx, x_t, v_t, dt)) != MLS_OK) return st;
  if ((st = contact_friction_lag(ctx)) != MLS_OK) return st;  // friction between bodies lagged at this x^t
  if ((st = launch_pack(ctx, x, ctx->xk)) != MLS_OK) return st;
  if ((st = assemble_at(ctx, ctx->xk, nullptr)) != MLS_OK) return st;
  if (grad_out && (st = launch_unpack(ctx, ctx->grad, grad_out)) != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "assemble sync");
}

mls_status mls_get_hessian(mls_ctx* ctx, int32_t* row_ptr, int32_t* colout, double* val, int64_t* nnzb) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  // with bodies, rows of surface vertices carry the contact blocks claimed at the last assembly
  const int* rl = ctx->h_row_len.data();
  const int* cl = ctx->h_col.data();
  std::vector<int> rl_dyn, col_dyn;
  int64_t nz = ctx->nnzb;
  if (ctx->cs.on && ctx->assembled) {
    rl_dyn.resize(ctx->n);
    col_dyn.resize((size_t)ctx->n_groups * kSlice);
    st = cuda_check(ctx, cudaMemcpy(rl_dyn.data(), ctx->row_len, sizeof(int) * ctx->n, cudaMemcpyDeviceToHost), "rows");
    if (st != MLS_OK) return st;
    st = cuda_check(ctx, cudaMemcpy(col_dyn.data(), ctx->col, sizeof(int) * col_dyn.size(), cudaMemcpyDeviceToHost),
                    "cols");
    if (st != MLS_OK) return st;
    rl = rl_dyn.data();
    cl = col_dyn.data();
    nz = 0;
    for (int v = 0; v < ctx->n; ++v) nz += rl[v];
  }
  if (nnzb) *nnzb = nz;
  if (!row_ptr && !colout && !val) return MLS_OK;
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "H not assembled");
  const int sb = storage_bytes(ctx);
  std::vector<unsigned char> raw((size_t)sb * 288 * ctx->n_groups);
  st = cuda_check(ctx, cudaMemcpy(raw.data(), ctx->hval, raw.size(), cudaMemcpyDeviceToHost), "H readback");
  if (st != MLS_OK) return st;
  int64_t pos = 0;
  for (int v = 0; v < ctx->n; ++v) {
    if (row_ptr) row_ptr[v] = (int32_t)pos;
    const int s = v / kSlice, lane = v % kSlice;
    // ascending column order for the exported CSR
    std::vector<std::pair<int, int>> order;
    for (int k = 0; k < rl[v]; ++k) order.emplace_back(cl[((size_t)ctx->h_slice_ptr[s] + k) * kSlice + lane], k);
    std::sort(order.begin(), order.end());
    for (auto& ck : order) {
      const int64_t g = (int64_t)ctx->h_slice_ptr[s] + ck.second;
      if (colout) colout[pos] = ck.first;
      if (val)
        for (int q = 0; q < 9; ++q) {
          const size_t idx = (size_t)g * 288 + q * 32 + lane;
          double x;
          if (sb == 8) x = ((const double*)raw.data())[idx];
          else if (sb == 4) x = ((const float*)raw.data())[idx];
          else {
            uint16_t b = ((const uint16_t*)raw.data())[idx];
            uint32_t u = (uint32_t)b << 16;
            float f;
            memcpy(&f, &u, 4);
            x = f;
          }
          val[pos * 9 + q] = x;
        }
      ++pos;
    }
  }
  if (row_ptr) row_ptr[ctx->n] = (int32_t)pos;
  return MLS_OK;
}

mls_status mls_spmv(mls_ctx* ctx, const double* x, double* y) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "H not assembled");
  if ((st = launch_pack(ctx, x, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_to_solve(ctx, ctx->dir, ctx->vp, 1.0)) != MLS_OK) return st;
  if ((st = launch_spmv(ctx, ctx->vp, ctx->vq)) != MLS_OK) return st;
  if ((st = launch_from_solve_raw(ctx, ctx->vq, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_unpack(ctx, ctx->dir, y)) != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "spmv sync");
}

mls_status mls_precond_apply(mls_ctx* ctx, const double* r, double* z) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "H not assembled");
  if ((st = launch_pack(ctx, r, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_to_solve(ctx, ctx->dir, ctx->vr, 1.0)) != MLS_OK) return st;
  if ((st = precond_apply(ctx, ctx->vr, ctx->vz)) != MLS_OK) return st;
  if ((st = launch_from_solve_raw(ctx, ctx->vz, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_unpack(ctx, ctx->dir, z)) != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "precond sync");
}

mls_status mls_pcg_solve(mls_ctx* ctx, const double* b, double* d, double rtol, int max_iter, int* iters,
                         double* rel_res) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->assembled) return fail(ctx, MLS_EINVAL, "H not assembled");
  if (!(rtol > 0) || max_iter < 1) return fail(ctx, MLS_EINVAL, "rtol must be > 0 and max_iter >= 1");
  if ((st = launch_pack(ctx, b, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_to_solve(ctx, ctx->dir, ctx->vb, 1.0)) != MLS_OK) return st;
  mls_status res = pcg_solve(ctx, rtol, max_iter, iters, rel_res);
  if (res != MLS_OK && res != MLS_ENOTCONV) return res;
  if ((st = launch_from_solve_raw(ctx, ctx->vx, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_unpack(ctx, ctx->dir, d)) != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "pcg sync");
  return st != MLS_OK ? st : res;
}

// q [m][12] float64 <-> solve precision on the device
__global__ void k_cast_in(int n, const double* __restrict__ a, float* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_cast_out(int n, const float* __restrict__ a, double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

mls_status mls_prolong(mls_ctx* ctx, const double* q, double* w) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  const int r = 12 * ctx->basis.m;
  if (ctx->opt.precision == MLS_FP64) {
    st = cuda_check(ctx, cudaMemcpyAsync(ctx->cvec, q, sizeof(double) * r, cudaMemcpyDeviceToDevice, ctx->stream), "q copy");
  } else {
    { ++ctx->launches; k_cast_in<<<(r + 255) / 256, 256, 0, ctx->stream>>>(r, q, (float*)ctx->cvec); }
    st = cuda_check(ctx, cudaGetLastError(), "cast");
  }
  if (st != MLS_OK) return st;
  if ((st = launch_prolong(ctx, ctx->cvec, ctx->vw, false)) != MLS_OK) return st;
  if ((st = launch_from_solve_raw(ctx, ctx->vw, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_unpack(ctx, ctx->dir, w)) != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "prolong sync");
}

mls_status mls_restrict(mls_ctx* ctx, const double* r, double* z) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  const int rr = 12 * ctx->basis.m;
  if ((st = launch_pack(ctx, r, ctx->dir)) != MLS_OK) return st;
  if ((st = launch_to_solve(ctx, ctx->dir, ctx->vr, 1.0)) != MLS_OK) return st;
  if ((st = launch_restrict(ctx, ctx->vr, ctx->cvec)) != MLS_OK) return st;
  if (ctx->opt.precision == MLS_FP64) {
    st = cuda_check(ctx, cudaMemcpyAsync(z, ctx->cvec, sizeof(double) * rr, cudaMemcpyDeviceToDevice, ctx->stream), "z copy");
  } else {
    { ++ctx->launches; k_cast_out<<<(rr + 255) / 256, 256, 0, ctx->stream>>>(rr, (const float*)ctx->cvec, z); }
    st = cuda_check(ctx, cudaGetLastError(), "cast");
  }
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "restrict sync");
}

mls_status mls_build_coarse(mls_ctx* ctx) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  st = build_coarse(ctx);
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "coarse sync");
}

mls_status mls_coarse_shift(mls_ctx* ctx, double* sigma) {
  if (!ctx || !sigma) return MLS_EINVAL;
  *sigma = ctx->coarse_sigma;
  return MLS_OK;
}

mls_status mls_get_coarse(mls_ctx* ctx, double* A) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!ctx->has_basis || !ctx->Acopy) return fail(ctx, MLS_EINVAL, "no coarse operator");
  const int r = 12 * ctx->basis.m;
  return cuda_check(ctx, cudaMemcpy(A, ctx->Acopy, sizeof(double) * r * r, cudaMemcpyDeviceToHost), "Ac readback");
}

mls_status mls_get_coarse_factor(mls_ctx* ctx, double* L) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!L) return fail(ctx, MLS_EINVAL, "null pointer");
  if (!ctx->has_basis || !ctx->coarse_ready || !ctx->Ac) return fail(ctx, MLS_EINVAL, "no coarse factor");
  const int r = 12 * ctx->basis.m;
  st = cuda_check(ctx, cudaMemcpy(L, ctx->Ac, sizeof(double) * r * r, cudaMemcpyDeviceToHost), "factor readback");
  if (st != MLS_OK) return st;
  for (int i = 0; i < r; ++i)
    for (int j = i + 1; j < r; ++j) L[(size_t)i * r + j] = 0.0;
  return MLS_OK;
}

mls_status mls_energy(mls_ctx* ctx, const double* x, const double* d, double alpha, double* E, int* feasible) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !d || !E) return fail(ctx, MLS_EINVAL, "null pointer");
  if ((st = launch_pack(ctx, x, ctx->xk)) != MLS_OK) return st;
  if ((st = launch_pack(ctx, d, ctx->dir)) != MLS_OK) return st;
  int inf = 0;
  if ((st = launch_energy(ctx, ctx->xk, ctx->dir, alpha, E, &inf)) != MLS_OK) return st;
  if (feasible) *feasible = inf ? 0 : 1;
  return MLS_OK;
}

mls_status mls_profile_enable(mls_ctx* ctx, uint32_t mask) {
  if (!ctx) return MLS_EINVAL;
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  else cudaDeviceSynchronize();
  ctx->prof_pending.clear();
  ctx->prof_mask = mask;
  for (int k = 0; k < MLS_PROF_COUNT; ++k) { ctx->prof_ms[k] = 0.0; ctx->prof_n[k] = 0; }
  return MLS_OK;
}

mls_status mls_profile_read(mls_ctx* ctx, double* ms, int64_t* launches) {
  if (!ctx) return MLS_EINVAL;
  mls_status st = cuda_check(ctx, ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize(), "profile sync");
  if (st != MLS_OK) return st;
  prof_flush(ctx);
  for (int k = 0; k < MLS_PROF_COUNT; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  return MLS_OK;
}

mls_status mls_ccd_bound(mls_ctx* ctx, const double* x, const double* d, double* alpha) {
  mls_status st = check_mesh(ctx);
  if (st != MLS_OK) return st;
  if (!x || !d || !alpha) return fail(ctx, MLS_EINVAL, "null pointer");
  if ((st = launch_pack(ctx, x, ctx->xk)) != MLS_OK) return st;
  if ((st = launch_pack(ctx, d, ctx->dir)) != MLS_OK) return st;
  return launch_ccd(ctx, ctx->xk, ctx->dir, alpha);
}

}  // extern "C"
