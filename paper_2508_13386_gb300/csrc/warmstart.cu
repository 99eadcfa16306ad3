// Learned warm start of the Newton loop from the coarse (SMS) state.
//
// Coarse coordinates of a configuration x are the mass-weighted projection
// onto the basis, q(x) = (U^T M U)^{-1} U^T M (x - X).  For each timestep the
// features are the coarse coordinates of the last two steps and of the
// external load, [q^t, q^{t-1}, q_g], with q_g the coarse coordinates of the
// gravity displacement h^2 g: q^t carries the deformation that sets the
// elastic force, q^t - q^{t-1} the velocity that sets x_tilde.  The target is the coarse
// Newton increment of the step: the Galerkin (H-orthogonal) projection
// dq = (U^T H U)^{-1} U^T H (x^{t+1} - x_tilde) with H and U^T H U taken at the
// step's first iterate, so that U dq is the best coarse approximation of the
// step in the energy norm and, when predicted well, x_tilde + U dq lowers E.
// With a trained network attached, the step starts from x_tilde + U dq_hat
// when that point is feasible and has lower energy than x_tilde, and from
// x_tilde otherwise (the plain start stays the fallback and the Newton/PCG
// solve the arbiter: the converged x^{t+1} does not depend on the start).
#include "mls_internal.cuh"

#include <cstring>

namespace mls {

mls_status factor_dense(mls_ctx* ctx, double* A, int r, double* Acopy, void* W, void* WT);
mls_status dense_apply(mls_ctx* ctx, const void* W, const void* WT, int r, const void* x, void* tmp, void* y);
mls_status mlp_forward_raw(mls_mlp* p, const float* X, int32_t batch, float* Y, cudaStream_t stream);
int mlp_width_in(const mls_mlp* p);
int mlp_width_out(const mls_mlp* p);

static inline int nb256(int64_t n) { return (int)((n + 255) / 256); }

// u_v = m_v (x_v - X_v) in solve precision
template <typename VT>
__global__ void k_mass_disp(int n, const double* __restrict__ mass, const Vec4d* __restrict__ x,
                            const Vec4d* __restrict__ X, Vec4<VT>* __restrict__ u) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const Vec4d a = x[v], b = X[v];
  const double m = mass[v];
  u[v] = Vec4<VT>{(VT)(m * (a.x - b.x)), (VT)(m * (a.y - b.y)), (VT)(m * (a.z - b.z)), VT(0)};
}

// u_v = m_v g h^2 (the gravity displacement, weighted)
template <typename VT>
__global__ void k_mass_const(int n, const double* __restrict__ mass, const uint8_t* __restrict__ pinned,
                             double gx, double gy, double gz, Vec4<VT>* __restrict__ u) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const double m = pinned[v] ? 0.0 : mass[v];
  u[v] = Vec4<VT>{(VT)(m * gx), (VT)(m * gy), (VT)(m * gz), VT(0)};
}

template <typename VT>
__global__ void k_to_double(int n, const VT* __restrict__ a, double* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

template <typename VT>
__global__ void k_from_float(int n, const float* __restrict__ a, VT* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (VT)a[i];
}

// features [q^t, q^{t-1}, qg] (float)
__global__ void k_features(int r, const double* __restrict__ hist, const double* __restrict__ qg,
                           float* __restrict__ f) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= r) return;
  f[i] = (float)hist[i];
  f[r + i] = (float)hist[r + i];
  f[2 * r + i] = (float)qg[i];
}

__global__ void k_diff_f(int r, const double* __restrict__ a, const double* __restrict__ b, float* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < r) out[i] = (float)(a[i] - b[i]);
}

__global__ void k_add_scaled4(int n, const Vec4d* __restrict__ a, const Vec4d* __restrict__ b, Vec4d* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Vec4d x = a[i], y = b[i];
  out[i] = Vec4d{x.x + y.x, x.y + y.y, x.z + y.z, 0.0};
}

// q(x) into q_out (float64 [r]); x float64 vertex vectors
mls_status coarse_project(mls_ctx* ctx, const Vec4d* x, double* q_out) {
  const int n = ctx->n, r = 12 * ctx->basis.m;
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_mass_disp<double><<<nb256(n), 256, 0, ctx->stream>>>(n, ctx->mass, x, ctx->X, (Vec4d*)ctx->vw); }
  } else {
    { ++ctx->launches; k_mass_disp<float><<<nb256(n), 256, 0, ctx->stream>>>(n, ctx->mass, x, ctx->X, (Vec4f*)ctx->vw); }
  }
  mls_status st = launch_restrict(ctx, ctx->vw, ctx->ws_c);
  if (st != MLS_OK) return st;
  if ((st = dense_apply(ctx, ctx->Wm, ctx->WmT, r, ctx->ws_c, ctx->ws_tmp, ctx->ws_c2)) != MLS_OK) return st;
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_to_double<double><<<nb256(r), 256, 0, ctx->stream>>>(r, (const double*)ctx->ws_c2, q_out); }
  } else {
    { ++ctx->launches; k_to_double<float><<<nb256(r), 256, 0, ctx->stream>>>(r, (const float*)ctx->ws_c2, q_out); }
  }
  return cuda_check(ctx, cudaGetLastError(), "coarse projection");
}

// U^T M U assembled on the host (12x12 blocks: I_3 (x) sum_v m_v phi_i phi_j a_i a_j^T)
// and factored on the device
mls_status warm_start_setup(mls_ctx* ctx) {
  const Basis& B = ctx->basis;
  const int m = B.m, r = 12 * m, n = ctx->n;
  mls_status st;
  if (!ctx->Am) {
    if ((st = dalloc(ctx, (void**)&ctx->Am, sizeof(double) * (size_t)r * r)) != MLS_OK) return st;
    const int vb = solve_bytes(ctx);
    if ((st = dalloc(ctx, &ctx->Wm, (size_t)vb * r * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->WmT, (size_t)vb * r * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->ws_c, (size_t)vb * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->ws_c2, (size_t)vb * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, &ctx->ws_tmp, (size_t)vb * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_hist, sizeof(double) * 3 * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_qg, sizeof(double) * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_qtilde, sizeof(double) * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_qnext, sizeof(double) * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_feat, sizeof(float) * 3 * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_target, sizeof(float) * r)) != MLS_OK) return st;
    if ((st = dalloc(ctx, (void**)&ctx->ws_pred, sizeof(float) * r)) != MLS_OK) return st;
  }
  std::vector<double> A((size_t)r * r, 0.0);
  for (int v = 0; v < n; ++v) {
    const double mv = ctx->h_mass[v];
    const double* Xv = &ctx->h_X[3 * (size_t)v];
    for (int p = B.h_vrow[v]; p < B.h_vrow[v + 1]; ++p) {
      const int i = B.h_vh[p];
      const double pi = B.h_vphi[p];
      const double ai[4] = {1.0, Xv[0] - B.h_origins[3 * i], Xv[1] - B.h_origins[3 * i + 1], Xv[2] - B.h_origins[3 * i + 2]};
      for (int q = B.h_vrow[v]; q < B.h_vrow[v + 1]; ++q) {
        const int j = B.h_vh[q];
        const double w = mv * pi * B.h_vphi[q];
        const double aj[4] = {1.0, Xv[0] - B.h_origins[3 * j], Xv[1] - B.h_origins[3 * j + 1], Xv[2] - B.h_origins[3 * j + 2]};
        for (int c = 0; c < 3; ++c)
          for (int l = 0; l < 4; ++l)
            for (int lp = 0; lp < 4; ++lp)
              A[(size_t)(12 * i + 4 * c + l) * r + 12 * j + 4 * c + lp] += w * ai[l] * aj[lp];
      }
    }
  }
  // handles without mass support keep an identity block so the factor exists
  for (int k = 0; k < r; ++k)
    if (A[(size_t)k * r + k] <= 0.0) A[(size_t)k * r + k] = 1.0;
  st = cuda_check(ctx, cudaMemcpy(ctx->Am, A.data(), sizeof(double) * A.size(), cudaMemcpyHostToDevice), "U^T M U upload");
  if (st != MLS_OK) return st;
  if ((st = factor_dense(ctx, ctx->Am, r, nullptr, ctx->Wm, ctx->WmT)) != MLS_OK) return st;
  // coarse coordinates of the gravity displacement h^2 g (h set at each step)
  ctx->ws_ready = true;
  ctx->ws_hist_valid = false;
  return MLS_OK;
}

static mls_status gravity_coords(mls_ctx* ctx) {
  const int n = ctx->n, r = 12 * ctx->basis.m;
  const double h2 = ctx->h * ctx->h;
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_mass_const<double><<<nb256(n), 256, 0, ctx->stream>>>(n, ctx->mass, ctx->pinned, h2 * ctx->grav[0], h2 * ctx->grav[1], h2 * ctx->grav[2], (Vec4d*)ctx->vw); }
  } else {
    { ++ctx->launches; k_mass_const<float><<<nb256(n), 256, 0, ctx->stream>>>(n, ctx->mass, ctx->pinned, h2 * ctx->grav[0], h2 * ctx->grav[1], h2 * ctx->grav[2], (Vec4f*)ctx->vw); }
  }
  mls_status st = launch_restrict(ctx, ctx->vw, ctx->ws_c);
  if (st != MLS_OK) return st;
  if ((st = dense_apply(ctx, ctx->Wm, ctx->WmT, r, ctx->ws_c, ctx->ws_tmp, ctx->ws_c2)) != MLS_OK) return st;
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_to_double<double><<<nb256(r), 256, 0, ctx->stream>>>(r, (const double*)ctx->ws_c2, ctx->ws_qg); }
  } else {
    { ++ctx->launches; k_to_double<float><<<nb256(r), 256, 0, ctx->stream>>>(r, (const float*)ctx->ws_c2, ctx->ws_qg); }
  }
  return cuda_check(ctx, cudaGetLastError(), "gravity coordinates");
}

// Called by the timestep after the predictor: updates the history with
// q(x^t), forms the features and, with a network attached, proposes the
// start x_tilde + U dq_hat (kept only when feasible with lower energy).
mls_status warm_start_begin(mls_ctx* ctx, int* used) {
  *used = 0;
  if (!ctx->ws_enabled || !ctx->ws_ready) return MLS_OK;
  const int r = 12 * ctx->basis.m;
  mls_status st;
  if ((st = coarse_project(ctx, ctx->xt, ctx->ws_qnext)) != MLS_OK) return st;
  if (!ctx->ws_hist_valid) {
    for (int k = 0; k < 3; ++k)
      if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->ws_hist + k * r, ctx->ws_qnext, sizeof(double) * r,
                                                cudaMemcpyDeviceToDevice, ctx->stream), "history")) != MLS_OK)
        return st;
    ctx->ws_hist_valid = true;
  } else {
    if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->ws_hist + r, ctx->ws_hist, sizeof(double) * 2 * r,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "history shift")) != MLS_OK)
      return st;
    if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->ws_hist, ctx->ws_qnext, sizeof(double) * r,
                                              cudaMemcpyDeviceToDevice, ctx->stream), "history")) != MLS_OK)
      return st;
  }
  if ((st = gravity_coords(ctx)) != MLS_OK) return st;
  { ++ctx->launches; k_features<<<nb256(r), 256, 0, ctx->stream>>>(r, ctx->ws_hist, ctx->ws_qg, ctx->ws_feat); }
  if (!ctx->ws_mlp) return cuda_check(ctx, cudaGetLastError(), "features");
  // prediction and candidate start
  if ((st = mlp_forward_raw(ctx->ws_mlp, ctx->ws_feat, 1, ctx->ws_pred, ctx->stream)) != MLS_OK)
    return fail(ctx, st, "warm start network forward");
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_from_float<double><<<nb256(r), 256, 0, ctx->stream>>>(r, ctx->ws_pred, (double*)ctx->ws_c); }
  } else {
    { ++ctx->launches; k_from_float<float><<<nb256(r), 256, 0, ctx->stream>>>(r, ctx->ws_pred, (float*)ctx->ws_c); }
  }
  if ((st = launch_prolong(ctx, ctx->ws_c, ctx->vw, false)) != MLS_OK) return st;
  if ((st = launch_from_solve(ctx, ctx->vw, ctx->dir)) != MLS_OK) return st;  // zero on Dirichlet vertices
  if (ctx->cs.on) {
    // Between bodies a feasible end point does not rule out a primitive that
    // passed through another on the way (Sec. 3.9): the candidate c is taken
    // only when the straight path x^t -> c, on which the start iterate is
    // cut too, needs no CCD cut, and when it lowers the energy of the start
    // the step has already chosen.
    if ((st = launch_axpy_state(ctx, ctx->dir, ctx->xtil, 1.0)) != MLS_OK) return st;
    if ((st = launch_axpy_state(ctx, ctx->dir, ctx->xt, -1.0)) != MLS_OK) return st;  // c - x^t
    double a = 0.0;
    if ((st = launch_ccd(ctx, ctx->xt, ctx->dir, &a)) != MLS_OK) return st;
    if (!(a >= 1.0)) return cuda_check(ctx, cudaGetLastError(), "warm start");
    double Ec = 0, Ecur = 0;
    int infc = 0, infcur = 0;
    if ((st = launch_energy(ctx, ctx->xk, ctx->tmp4, 0.0, &Ecur, &infcur)) != MLS_OK) return st;
    if ((st = launch_energy(ctx, ctx->xt, ctx->dir, 1.0, &Ec, &infc)) != MLS_OK) return st;
    if (!infc && std::isfinite(Ec) && (infcur || Ec < Ecur)) {
      if ((st = launch_xpay_state(ctx, ctx->xt, ctx->dir, 1.0, ctx->xk)) != MLS_OK) return st;
      *used = 1;
    }
    return cuda_check(ctx, cudaGetLastError(), "warm start");
  }
  double E0 = 0, E1 = 0;
  int inf0 = 0, inf1 = 0;
  if ((st = launch_energy(ctx, ctx->xtil, ctx->dir, 0.0, &E0, &inf0)) != MLS_OK) return st;
  if ((st = launch_energy(ctx, ctx->xtil, ctx->dir, 1.0, &E1, &inf1)) != MLS_OK) return st;
  if (!inf1 && (inf0 || E1 < E0)) {
    { ++ctx->launches; k_add_scaled4<<<nb256(ctx->n), 256, 0, ctx->stream>>>(ctx->n, ctx->xtil, ctx->dir, ctx->xk); }
    *used = 1;
  }
  return cuda_check(ctx, cudaGetLastError(), "warm start");
}

template <typename VT>
__global__ void k_to_float(int n, const VT* __restrict__ a, float* __restrict__ b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

__global__ void k_sub4(int n, const Vec4d* __restrict__ a, const Vec4d* __restrict__ b, Vec4d* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Vec4d x = a[i], y = b[i];
  out[i] = Vec4d{x.x - y.x, x.y - y.y, x.z - y.z, 0.0};
}

// After the first Newton iteration's assembly (and coarse build): keep H(x_tilde)
mls_status warm_start_first_iteration(mls_ctx* ctx) {
  if (!ctx->ws_enabled || !ctx->ws_record) return MLS_OK;
  const size_t bytes = (size_t)storage_bytes(ctx) * 288 * ctx->n_groups;
  if (!ctx->ws_hsave) {
    mls_status st = dalloc(ctx, &ctx->ws_hsave, bytes);
    if (st != MLS_OK) return st;
  }
  return cuda_check(ctx, cudaMemcpyAsync(ctx->ws_hsave, ctx->hval, bytes, cudaMemcpyDeviceToDevice, ctx->stream),
                    "H copy");
}

// Called after the Newton loop when recording: the target
// (U^T H U)^{-1} U^T H (x^{t+1} - x_tilde) at the first iterate
mls_status warm_start_end(mls_ctx* ctx) {
  if (!ctx->ws_enabled || !ctx->ws_ready || !ctx->ws_record || !ctx->ws_hsave || !ctx->coarse_ready) return MLS_OK;
  const int n = ctx->n, r = 12 * ctx->basis.m;
  { ++ctx->launches; k_sub4<<<nb256(n), 256, 0, ctx->stream>>>(n, ctx->xk, ctx->xtil, ctx->tmp4); }
  mls_status st = launch_to_solve(ctx, ctx->tmp4, ctx->vb, 1.0);
  if (st != MLS_OK) return st;
  // tmp4 is the library's zero vector between calls: restore it
  if ((st = cuda_check(ctx, cudaMemsetAsync(ctx->tmp4, 0, sizeof(Vec4d) * n, ctx->stream), "zero")) != MLS_OK) return st;
  if ((st = launch_spmv_values(ctx, ctx->ws_hsave, ctx->vb, ctx->vq)) != MLS_OK) return st;
  if ((st = launch_restrict(ctx, ctx->vq, ctx->ws_c)) != MLS_OK) return st;
  if ((st = coarse_apply(ctx, ctx->ws_c, ctx->ws_c2)) != MLS_OK) return st;
  if (ctx->opt.precision == MLS_FP64) {
    { ++ctx->launches; k_to_float<double><<<nb256(r), 256, 0, ctx->stream>>>(r, (const double*)ctx->ws_c2, ctx->ws_target); }
  } else {
    { ++ctx->launches; k_to_float<float><<<nb256(r), 256, 0, ctx->stream>>>(r, (const float*)ctx->ws_c2, ctx->ws_target); }
  }
  return cuda_check(ctx, cudaGetLastError(), "warm start target");
}

}  // namespace mls

using namespace mls;

extern "C" {

mls_status mls_warm_start_enable(mls_ctx* ctx, int enable) {
  if (!ctx || enable < 0 || enable > 2) return MLS_EINVAL;
  if (!enable) {
    ctx->ws_enabled = false;
    ctx->ws_record = false;
    return MLS_OK;
  }
  if (enable == 2 && ctx->opt.preconditioner != MLS_PRECOND_TWO_LEVEL)
    return fail(ctx, MLS_EINVAL, "recording targets needs the two-level preconditioner (its coarse factor)");
  ctx->ws_record = (enable == 2);
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "warm start needs an uploaded basis");
  if (!ctx->ws_ready) {
    mls_status st = warm_start_setup(ctx);
    if (st != MLS_OK) return st;
  }
  ctx->ws_enabled = true;
  ctx->ws_hist_valid = false;
  return MLS_OK;
}

mls_status mls_warm_start_reset(mls_ctx* ctx) {
  if (!ctx) return MLS_EINVAL;
  ctx->ws_hist_valid = false;
  return MLS_OK;
}

mls_status mls_warm_start_attach(mls_ctx* ctx, mls_mlp* mlp) {
  if (!ctx) return MLS_EINVAL;
  if (mlp) {
    const int r = 12 * ctx->basis.m;
    if (!ctx->has_basis || mlp_width_in(mlp) != 3 * r || mlp_width_out(mlp) != r)
      return fail(ctx, MLS_EINVAL, "network widths must be 3 r inputs and r outputs (r = 12 handles)");
  }
  ctx->ws_mlp = mlp;
  return MLS_OK;
}

mls_status mls_warm_start_sample(mls_ctx* ctx, float* features, float* target) {
  if (!ctx || !features || !target) return MLS_EINVAL;
  if (!ctx->ws_enabled || !ctx->ws_ready) return fail(ctx, MLS_EINVAL, "warm start is not enabled");
  const int r = 12 * ctx->basis.m;
  mls_status st = cuda_check(ctx, cudaMemcpyAsync(features, ctx->ws_feat, sizeof(float) * 3 * r,
                                                  cudaMemcpyDeviceToDevice, ctx->stream), "features");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(target, ctx->ws_target, sizeof(float) * r, cudaMemcpyDeviceToDevice,
                                       ctx->stream), "target");
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "sample sync");
}

mls_status mls_coarse_project(mls_ctx* ctx, const double* x, double* q) {
  if (!ctx || !x || !q) return MLS_EINVAL;
  if (!ctx->has_basis) return fail(ctx, MLS_EINVAL, "no basis uploaded");
  if (!ctx->ws_ready) {
    mls_status st = warm_start_setup(ctx);
    if (st != MLS_OK) return st;
  }
  mls_status st = launch_pack(ctx, x, ctx->dir);
  if (st != MLS_OK) return st;
  if ((st = coarse_project(ctx, ctx->dir, q)) != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "projection sync");
}

}  // extern "C"
