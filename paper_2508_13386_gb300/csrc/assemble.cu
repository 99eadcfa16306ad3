// Gradient and Hessian assembly of the incremental potential (Eq. IP with
// implicit Euler, Sec. 3.1), and the state-vector helpers of the timestep.
//
//   g = M (x - x_tilde) + h^2 (sum_e grad_e + kappa b'(d_v) n + grad D_v),
//       g_v = 0 on Dirichlet vertices;
//   H = M + h^2 (sum_e H_e + kappa b''(d_v) n n^T + hess D_v), Dirichlet rows
//       and columns replaced by the identity.
// D_v is the lagged point-plane friction (zero unless a friction coefficient
// is set).  With BDF2 the same forms hold with h = 2/3 of the timestep and
// the BDF2 predictor x_tilde.
//
// Both are deterministic gathers (no floating-point atomics): every vertex
// sums its incident element gradients through a precomputed incidence list
// and every block slot of H sums the element blocks mapped onto it.
#include "mls_internal.cuh"

namespace mls {

struct AsmIn {
  int n, t;
  const double* __restrict__ mass;
  const uint8_t* __restrict__ pinned;
  const Vec4d* __restrict__ xtil;
  const int* __restrict__ vt_ptr;
  const int* __restrict__ vt_code;
  const double* __restrict__ egrad;
  double h2, kappa, dhat, po, pn0, pn1, pn2;
  int contact;
  const Vec4d* __restrict__ xt;  // x^t, the friction lag state
  double fmu, feps;              // friction coefficient (0: none) and mollifier width
  const Vec4d* __restrict__ cgrad;  // mesh-mesh barrier gradient per vertex (nullable)
};

__device__ __forceinline__ double bar_db(double d, double dhat) {
  if (d >= dhat || d <= 0.0) return 0.0;
  const double r = d - dhat;
  return -2.0 * r * log(d / dhat) - r * r / d;
}
__device__ __forceinline__ double bar_d2b(double d, double dhat) {
  if (d >= dhat || d <= 0.0) return 0.0;
  const double r = d - dhat;
  return -2.0 * log(d / dhat) - 4.0 * r / d + r * r / (d * d);
}

// g (float64) and the PCG right-hand side b = -g in solve precision; FRIC
// compiles the friction term in (the instance without it is the plain kernel)
template <typename VT, bool FRIC>
__global__ void __launch_bounds__(kBlock) k_gather_grad(AsmIn in, const Vec4d* __restrict__ x,
                                                        Vec4d* __restrict__ g, Vec4<VT>* __restrict__ b,
                                                        GridReduce gr, double* __restrict__ gnorm2) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (v < in.n) {
    Vec4d gv{0.0, 0.0, 0.0, 0.0};
    if (!in.pinned[v]) {
      double sx = 0.0, sy = 0.0, sz = 0.0;
      const int t = in.t;
      for (int k = in.vt_ptr[v]; k < in.vt_ptr[v + 1]; ++k) {
        const int code = in.vt_code[k];
        const int e = code >> 2, a = code & 3;
        sx += in.egrad[(3 * a + 0) * t + e];
        sy += in.egrad[(3 * a + 1) * t + e];
        sz += in.egrad[(3 * a + 2) * t + e];
      }
      const Vec4d xv = x[v];
      if (in.contact) {
        const double dist = in.pn0 * xv.x + in.pn1 * xv.y + in.pn2 * xv.z - in.po;
        const double k1 = in.kappa * bar_db(dist, in.dhat);
        sx += k1 * in.pn0; sy += k1 * in.pn1; sz += k1 * in.pn2;
        if constexpr (FRIC) {
          const Vec4d xtv = in.xt[v];
          const double lam = fric_lambda(in.pn0 * xtv.x + in.pn1 * xtv.y + in.pn2 * xtv.z - in.po, in.dhat,
                                         in.kappa);
          if (lam > 0.0) {
            double u[3];
            const double y = fric_slip(xv, xtv, in.pn0, in.pn1, in.pn2, u);
            const double f = in.fmu * lam * fric_ratio(y, in.feps);
            sx += f * u[0]; sy += f * u[1]; sz += f * u[2];
          }
        }
      }
      if (in.cgrad) {
        const Vec4d cg = in.cgrad[v];
        sx += cg.x; sy += cg.y; sz += cg.z;
      }
      const Vec4d xt = in.xtil[v];
      const double m = in.mass[v];
      gv.x = m * (xv.x - xt.x) + in.h2 * sx;
      gv.y = m * (xv.y - xt.y) + in.h2 * sy;
      gv.z = m * (xv.z - xt.z) + in.h2 * sz;
    }
    g[v] = gv;
    b[v] = Vec4<VT>{(VT)(-gv.x), (VT)(-gv.y), (VT)(-gv.z), (VT)0};
    acc[0] = gv.x * gv.x + gv.y * gv.y + gv.z * gv.z;
  }
  if (grid_sum<1>(acc, gr, RS_GRAD) && threadIdx.x == 0) *gnorm2 = acc[0];
}

struct SellAsmIn {
  int n, t;
  const int* __restrict__ group_slice;
  const int* __restrict__ col;
  const int* __restrict__ row_len;
  const int* __restrict__ slice_ptr;
  const int* __restrict__ asm_ptr;
  const int* __restrict__ asm_code;
  const double* __restrict__ mass;
  const uint8_t* __restrict__ pinned;
  double h2, kappa, dhat, po, pn0, pn1, pn2;
  int contact;
  const Vec4d* __restrict__ xt;  // x^t, the friction lag state
  double fmu, feps;              // friction coefficient (0: none) and mollifier width
};

template <typename AT, typename ET>
__device__ __forceinline__ void add_elem_block(AT (&acc)[9], const ET* __restrict__ hs, int t, int e,
                                               int a, int b) {
  if (a == b) {
    const int off = hess_offset(a, a);
    const AT h00 = load_as<AT>(hs[(off + 0) * t + e]), h01 = load_as<AT>(hs[(off + 1) * t + e]),
             h02 = load_as<AT>(hs[(off + 2) * t + e]), h11 = load_as<AT>(hs[(off + 3) * t + e]),
             h12 = load_as<AT>(hs[(off + 4) * t + e]), h22 = load_as<AT>(hs[(off + 5) * t + e]);
    acc[0] += h00; acc[1] += h01; acc[2] += h02;
    acc[3] += h01; acc[4] += h11; acc[5] += h12;
    acc[6] += h02; acc[7] += h12; acc[8] += h22;
  } else if (a < b) {
    const int off = hess_offset(a, b);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] += load_as<AT>(hs[(off + k) * t + e]);
  } else {
    const int off = hess_offset(b, a);
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int d = 0; d < 3; ++d) acc[3 * c + d] += load_as<AT>(hs[(off + 3 * d + c) * t + e]);
  }
}

template <typename T>
__device__ __forceinline__ void inv3(const T (&A)[9], T (&R)[9]) {
  const T c00 = A[4] * A[8] - A[5] * A[7];
  const T c01 = A[5] * A[6] - A[3] * A[8];
  const T c02 = A[3] * A[7] - A[4] * A[6];
  const T det = A[0] * c00 + A[1] * c01 + A[2] * c02;
  const T id = T(1) / det;
  R[0] = c00 * id;
  R[1] = (A[2] * A[7] - A[1] * A[8]) * id;
  R[2] = (A[1] * A[5] - A[2] * A[4]) * id;
  R[3] = c01 * id;
  R[4] = (A[0] * A[8] - A[2] * A[6]) * id;
  R[5] = (A[2] * A[3] - A[0] * A[5]) * id;
  R[6] = c02 * id;
  R[7] = (A[1] * A[6] - A[0] * A[7]) * id;
  R[8] = (A[0] * A[4] - A[1] * A[3]) * id;
}

// One thread per block slot of H.  AT: accumulation type, ET: element
// Hessian type, MT: storage type of H, VT: solve type (for D^{-1}).
// escale (nullable): a factor per element on its elastic Hessian (a
// cubature of the elastic term, Sec. 3.8; mass and barrier stay whole).
// dinv (nullable): the block-Jacobi inverse of the stored diagonal blocks.
// FRIC compiles the friction blocks in (the instance without it is the plain kernel).
template <typename AT, typename ET, typename MT, typename VT, bool FRIC>
__global__ void __launch_bounds__(kBlock) k_assemble(SellAsmIn in, int64_t n_slots,
                                                     const Vec4d* __restrict__ x,
                                                     const ET* __restrict__ hs, MT* __restrict__ val,
                                                     VT* __restrict__ dinv, const double* __restrict__ escale) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_slots) return;
  const int64_t g = s >> 5;
  const int lane = (int)(s & 31);
  const int slice = in.group_slice[g];
  const int row = slice * kSlice + lane;
  if (row >= in.n) return;
  const int k = (int)(g - in.slice_ptr[slice]);
  MT* out = val + g * 288 + lane;
  if (k >= in.row_len[row]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) out[q * 32] = from_d<MT>(0.0);
    return;
  }
  const int c = in.col[s];
  AT acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = AT(0);
  const bool pin = in.pinned[row] || in.pinned[c];
  if (pin) {
    if (c == row) { acc[0] = AT(1); acc[4] = AT(1); acc[8] = AT(1); }
  } else {
    for (int q = in.asm_ptr[s]; q < in.asm_ptr[s + 1]; ++q) {
      const int code = in.asm_code[q];
      if (escale) {
        const double se = escale[code >> 4];
        if (se == 0.0) continue;
        AT part[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) part[k] = AT(0);
        add_elem_block<AT, ET>(part, hs, in.t, code >> 4, (code >> 2) & 3, code & 3);
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += (AT)se * part[k];
      } else {
        add_elem_block<AT, ET>(acc, hs, in.t, code >> 4, (code >> 2) & 3, code & 3);
      }
    }
    const AT h2 = (AT)in.h2;
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] *= h2;
    if (c == row) {
      const AT m = (AT)in.mass[row];
      acc[0] += m; acc[4] += m; acc[8] += m;
      if (in.contact) {
        const Vec4d xv = x[row];
        const double dist = in.pn0 * xv.x + in.pn1 * xv.y + in.pn2 * xv.z - in.po;
        const double k2 = in.h2 * in.kappa * bar_d2b(dist, in.dhat);
        if (k2 != 0.0) {
          const double nn[3] = {in.pn0, in.pn1, in.pn2};
#pragma unroll
          for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) acc[3 * a + b] += (AT)(k2 * nn[a] * nn[b]);
        }
        if constexpr (FRIC) {
          const Vec4d xtv = in.xt[row];
          const double lam = fric_lambda(in.pn0 * xtv.x + in.pn1 * xtv.y + in.pn2 * xtv.z - in.po, in.dhat,
                                         in.kappa);
          if (lam > 0.0) {
            double u[3];
            const double y = fric_slip(xv, xtv, in.pn0, in.pn1, in.pn2, u);
            const double w = in.h2 * in.fmu * lam;
            const double r = fric_ratio(y, in.feps);
            // (slope - ratio) u^ u^T; at y = 0 the two factors are equal and the term vanishes
            const double su = y > 0.0 ? fric_slope(y, in.feps) - r : 0.0;
            const double iy = y > 0.0 ? 1.0 / y : 0.0;
            const double uh[3] = {u[0] * iy, u[1] * iy, u[2] * iy};
            const double nn[3] = {in.pn0, in.pn1, in.pn2};
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
              for (int b = 0; b < 3; ++b)
                acc[3 * a + b] += (AT)(w * (r * ((a == b ? 1.0 : 0.0) - nn[a] * nn[b]) + su * uh[a] * uh[b]));
          }
        }
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) out[q * 32] = from_d<MT>((double)acc[q]);
  if (c == row && dinv) {
    // block-Jacobi inverse of the diagonal block as stored
    VT A[9], R[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) A[q] = load_as<VT>(from_d<MT>((double)acc[q]));
    inv3<VT>(A, R);
#pragma unroll
    for (int q = 0; q < 9; ++q) dinv[(int64_t)row * 9 + q] = R[q];
  }
}

// ---- state helpers ------------------------------------------------------------------
__global__ void k_predictor(int n, const double* __restrict__ x, const double* __restrict__ v,
                            const uint8_t* __restrict__ pinned, double h, double gx, double gy,
                            double gz, Vec4d* __restrict__ xt, Vec4d* __restrict__ xtil,
                            Vec4d* __restrict__ xk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Vec4d p{x[3 * i], x[3 * i + 1], x[3 * i + 2], 0.0};
  xt[i] = p;
  Vec4d q = p;
  if (!pinned[i]) {
    const double h2 = h * h;
    q.x = p.x + h * v[3 * i] + h2 * gx;
    q.y = p.y + h * v[3 * i + 1] + h2 * gy;
    q.z = p.z + h * v[3 * i + 2] + h2 * gz;
  }
  xtil[i] = q;
  xk[i] = q;
}

// BDF2 predictor (Sec. 3.1): x_tilde = (4 x^t - x^{t-1}) / 3 + (2h/9)(4 v^t - v^{t-1})
// + (4/9) h^2 g on free vertices, x^t on Dirichlet vertices; h is the timestep
__global__ void k_predictor_bdf2(int n, const double* __restrict__ x, const double* __restrict__ v,
                                 const double* __restrict__ xp, const double* __restrict__ vp,
                                 const uint8_t* __restrict__ pinned, double h, double gx, double gy, double gz,
                                 Vec4d* __restrict__ xt, Vec4d* __restrict__ xtil, Vec4d* __restrict__ xk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const Vec4d p{x[3 * i], x[3 * i + 1], x[3 * i + 2], 0.0};
  xt[i] = p;
  Vec4d q = p;
  if (!pinned[i]) {
    const double a = 2.0 * h / 9.0, b = 4.0 * h * h / 9.0;
    q.x = (4.0 * p.x - xp[3 * i]) / 3.0 + a * (4.0 * v[3 * i] - vp[3 * i]) + b * gx;
    q.y = (4.0 * p.y - xp[3 * i + 1]) / 3.0 + a * (4.0 * v[3 * i + 1] - vp[3 * i + 1]) + b * gy;
    q.z = (4.0 * p.z - xp[3 * i + 2]) / 3.0 + a * (4.0 * v[3 * i + 2] - vp[3 * i + 2]) + b * gz;
  }
  xtil[i] = q;
  xk[i] = q;
}

__global__ void k_pack(int n, const double* __restrict__ src, Vec4d* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = Vec4d{src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.0};
}

__global__ void k_unpack(int n, const Vec4d* __restrict__ src, double* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4d s = src[i];
    dst[3 * i] = s.x; dst[3 * i + 1] = s.y; dst[3 * i + 2] = s.z;
  }
}

__global__ void k_disp(int n, const Vec4d* __restrict__ xk, const Vec4d* __restrict__ xt,
                       double* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4d a = xk[i], b = xt[i];
    dx[3 * i] = a.x - b.x; dx[3 * i + 1] = a.y - b.y; dx[3 * i + 2] = a.z - b.z;
  }
}

__global__ void k_axpy_state(int n, Vec4d* __restrict__ x, const Vec4d* __restrict__ d, double alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    Vec4d a = x[i];
    const Vec4d b = d[i];
    a.x += alpha * b.x; a.y += alpha * b.y; a.z += alpha * b.z;
    x[i] = a;
  }
}

template <typename VT>
__global__ void k_to_solve(int n, const Vec4d* __restrict__ src, Vec4<VT>* __restrict__ dst, double scale) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4d s = src[i];
    dst[i] = Vec4<VT>{(VT)(scale * s.x), (VT)(scale * s.y), (VT)(scale * s.z), (VT)0};
  }
}

template <typename VT>
__global__ void k_from_solve(int n, const Vec4<VT>* __restrict__ src, const uint8_t* __restrict__ pinned,
                             Vec4d* __restrict__ dst) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4<VT> s = src[i];
    dst[i] = (pinned && pinned[i]) ? Vec4d{0.0, 0.0, 0.0, 0.0} : Vec4d{(double)s.x, (double)s.y, (double)s.z, 0.0};
  }
}

template <typename VT>
__global__ void k_add_solve(int n, Vec4<VT>* __restrict__ y, const Vec4<VT>* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    Vec4<VT> a = y[i];
    const Vec4<VT> b = x[i];
    a.x += b.x; a.y += b.y; a.z += b.z;
    y[i] = a;
  }
}

__global__ void k_diff_state(int n, const Vec4d* __restrict__ a, const Vec4d* __restrict__ b, Vec4d* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4d p = a[i], q = b[i];
    out[i] = Vec4d{p.x - q.x, p.y - q.y, p.z - q.z, 0.0};
  }
}

__global__ void k_xpay_state(int n, const Vec4d* __restrict__ x, const Vec4d* __restrict__ d, double alpha,
                             Vec4d* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const Vec4d p = x[i], q = d[i];
    out[i] = Vec4d{p.x + alpha * q.x, p.y + alpha * q.y, p.z + alpha * q.z, 0.0};
  }
}

// ---- launchers -----------------------------------------------------------------------
static AsmIn asm_in(mls_ctx* ctx) {
  return AsmIn{ctx->n, ctx->t, ctx->mass, ctx->pinned, ctx->xtil, ctx->vt_ptr, ctx->vt_code, ctx->egrad,
               ctx->h * ctx->h, ctx->kappa, ctx->dhat, ctx->po, ctx->pn[0], ctx->pn[1], ctx->pn[2],
               ctx->contact, ctx->xt, ctx->contact ? ctx->fric_mu : 0.0, ctx->fric_eps_v * ctx->h_step,
               ctx->cs.on ? ctx->cs.cgrad : nullptr};
}

static inline int nblk(int64_t n, int b = kBlock) { return (int)((n + b - 1) / b); }

mls_status launch_gather_grad(mls_ctx* ctx, const Vec4d* x, double* gnorm2_out) {
  const int nb = nblk(ctx->n);
  if (nb > kMaxPartials) return fail(ctx, MLS_EINVAL, "mesh too large for one reduction grid");
  const AsmIn in = asm_in(ctx);
  const bool fric = in.fmu > 0.0;
  ++ctx->launches;
  if (ctx->opt.precision == MLS_FP64) {
    if (fric) k_gather_grad<double, true><<<nb, kBlock, 0, ctx->stream>>>(in, x, ctx->grad, (Vec4d*)ctx->vb, ctx->red, gnorm2_out);
    else k_gather_grad<double, false><<<nb, kBlock, 0, ctx->stream>>>(in, x, ctx->grad, (Vec4d*)ctx->vb, ctx->red, gnorm2_out);
  } else {
    if (fric) k_gather_grad<float, true><<<nb, kBlock, 0, ctx->stream>>>(in, x, ctx->grad, (Vec4f*)ctx->vb, ctx->red, gnorm2_out);
    else k_gather_grad<float, false><<<nb, kBlock, 0, ctx->stream>>>(in, x, ctx->grad, (Vec4f*)ctx->vb, ctx->red, gnorm2_out);
  }
  return cuda_check(ctx, cudaGetLastError(), "k_gather_grad");
}

// H (or, with escale, the cubature H of the coarse operator) at x into val;
// dinv (nullable) receives the block-Jacobi inverse
static mls_status assemble_into(mls_ctx* ctx, const Vec4d* x, const void* eh, void* val, void* dinv,
                                const double* escale) {
  SellAsmIn in{ctx->n, ctx->t, ctx->group_slice, ctx->col, ctx->row_len, ctx->slice_ptr, ctx->asm_ptr,
               ctx->asm_code, ctx->mass, ctx->pinned, ctx->h * ctx->h, ctx->kappa, ctx->dhat, ctx->po,
               ctx->pn[0], ctx->pn[1], ctx->pn[2], ctx->contact, ctx->xt,
               ctx->contact ? ctx->fric_mu : 0.0, ctx->fric_eps_v * ctx->h_step};
  const int64_t n_slots = ctx->n_groups * kSlice;
  const int nb = nblk(n_slots);
  const bool fric = in.fmu > 0.0;
  ++ctx->launches;
  switch (ctx->opt.precision) {
    case MLS_FP64:
      if (fric)
        k_assemble<double, double, double, double, true><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const double*)eh, (double*)val, (double*)dinv, escale);
      else
        k_assemble<double, double, double, double, false><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const double*)eh, (double*)val, (double*)dinv, escale);
      break;
    case MLS_MIXED_FP32:
      if (fric)
        k_assemble<float, float, float, float, true><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const float*)eh, (float*)val, (float*)dinv, escale);
      else
        k_assemble<float, float, float, float, false><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const float*)eh, (float*)val, (float*)dinv, escale);
      break;
    default:
      if (fric)
        k_assemble<float, float, __nv_bfloat16, float, true><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const float*)eh, (__nv_bfloat16*)val, (float*)dinv, escale);
      else
        k_assemble<float, float, __nv_bfloat16, float, false><<<nb, kBlock, 0, ctx->stream>>>(
            in, n_slots, x, (const float*)eh, (__nv_bfloat16*)val, (float*)dinv, escale);
      break;
  }
  return cuda_check(ctx, cudaGetLastError(), "k_assemble");
}

mls_status launch_assemble(mls_ctx* ctx, const Vec4d* x) {
  return assemble_into(ctx, x, ctx->ehess, ctx->hval, ctx->dinv, nullptr);
}

mls_status launch_assemble_cubature(mls_ctx* ctx, const Vec4d* x) {
  if (!ctx->cub_scale || !ctx->hval_cub) return fail(ctx, MLS_EINVAL, "no cubature uploaded");
  mls_status st = assemble_into(ctx, x, ctx->ehess, ctx->hval_cub, nullptr, ctx->cub_scale);
  if (st != MLS_OK) return st;
  return contact_merge(ctx, ctx->hval_cub, nullptr, false);
}

// H_lag of the paper's refinement (Sec. 3.7.2): the element Hessians saved at
// the last refresh with the mass and the contact and friction blocks of x
mls_status launch_assemble_lagged(mls_ctx* ctx, const Vec4d* x) {
  mls_status st = assemble_into(ctx, x, ctx->ehess_lag, ctx->hval_lag, ctx->dinv_lag, nullptr);
  if (st != MLS_OK) return st;
  return contact_merge(ctx, ctx->hval_lag, ctx->dinv_lag, false);
}

mls_status launch_predictor(mls_ctx* ctx, const double* x, const double* v, double dt) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_predictor<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, x, v, ctx->pinned, dt, ctx->grav[0],
                                                       ctx->grav[1], ctx->grav[2], ctx->xt, ctx->xtil,
                                                       ctx->xk); }
  return cuda_check(ctx, cudaGetLastError(), "k_predictor");
}

mls_status launch_predictor_bdf2(mls_ctx* ctx, const double* x, const double* v, const double* x_prev,
                                 const double* v_prev, double dt) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_predictor_bdf2<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(
        ctx->n, x, v, x_prev, v_prev, ctx->pinned, dt, ctx->grav[0], ctx->grav[1], ctx->grav[2], ctx->xt,
        ctx->xtil, ctx->xk); }
  return cuda_check(ctx, cudaGetLastError(), "k_predictor_bdf2");
}

mls_status launch_pack(mls_ctx* ctx, const double* src, Vec4d* dst) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_pack<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, src, dst); }
  return cuda_check(ctx, cudaGetLastError(), "k_pack");
}

mls_status launch_unpack(mls_ctx* ctx, const Vec4d* src, double* dst) {
  { ++ctx->launches; k_unpack<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, src, dst); }
  return cuda_check(ctx, cudaGetLastError(), "k_unpack");
}

mls_status launch_disp_out(mls_ctx* ctx, double* dx_out) {
  { ++ctx->launches; k_disp<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, ctx->xk, ctx->xt, dx_out); }
  return cuda_check(ctx, cudaGetLastError(), "k_disp");
}

mls_status launch_axpy_state(mls_ctx* ctx, Vec4d* x, const Vec4d* d, double alpha) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_axpy_state<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, x, d, alpha); }
  return cuda_check(ctx, cudaGetLastError(), "k_axpy_state");
}

mls_status launch_diff_state(mls_ctx* ctx, const Vec4d* a, const Vec4d* b, Vec4d* out) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_diff_state<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, a, b, out); }
  return cuda_check(ctx, cudaGetLastError(), "k_diff_state");
}

mls_status launch_xpay_state(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, Vec4d* out) {
  contact_invalidate(ctx);
  { ++ctx->launches; k_xpay_state<<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, x, d, alpha, out); }
  return cuda_check(ctx, cudaGetLastError(), "k_xpay_state");
}

mls_status launch_to_solve(mls_ctx* ctx, const Vec4d* src, void* dst, double scale) {
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_to_solve<double><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, src, (Vec4d*)dst, scale); }
  else
    { ++ctx->launches; k_to_solve<float><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, src, (Vec4f*)dst, scale); }
  return cuda_check(ctx, cudaGetLastError(), "k_to_solve");
}

mls_status launch_add_solve(mls_ctx* ctx, void* y, const void* x) {
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_add_solve<double><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (Vec4d*)y, (const Vec4d*)x); }
  else
    { ++ctx->launches; k_add_solve<float><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (Vec4f*)y, (const Vec4f*)x); }
  return cuda_check(ctx, cudaGetLastError(), "k_add_solve");
}

mls_status launch_from_solve(mls_ctx* ctx, const void* src, Vec4d* dst) {
  contact_invalidate(ctx);
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_from_solve<double><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const Vec4d*)src, ctx->pinned, dst); }
  else
    { ++ctx->launches; k_from_solve<float><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const Vec4f*)src, ctx->pinned, dst); }
  return cuda_check(ctx, cudaGetLastError(), "k_from_solve");
}

mls_status launch_from_solve_raw(mls_ctx* ctx, const void* src, Vec4d* dst) {
  contact_invalidate(ctx);
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_from_solve<double><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const Vec4d*)src, nullptr, dst); }
  else
    { ++ctx->launches; k_from_solve<float><<<nblk(ctx->n), kBlock, 0, ctx->stream>>>(ctx->n, (const Vec4f*)src, nullptr, dst); }
  return cuda_check(ctx, cudaGetLastError(), "k_from_solve");
}

}  // namespace mls
