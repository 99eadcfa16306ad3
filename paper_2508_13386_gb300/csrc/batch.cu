// Batched timestep: many independent meshes advanced together.
//
// Every mesh of the batch runs its own projected Newton loop on the
// incremental potential (Sec. 3.1, Eq. 5) with a block-Jacobi PCG solve and
// the filtered backtracking line search (Sec. 3.9) -- the same iteration as
// the single-mesh timestep, with its own scalars, tolerances and stopping
// decisions per mesh.  The meshes are stored as one concatenated mesh (their
// Hessian is block diagonal), each mesh's vertex range padded with pinned
// dummy vertices to whole 32-row slices, so that every SELL slice, every
// row block and every tet block belongs to exactly one mesh.
//
// Control lives on the device.  Per-mesh reductions use block partials
// summed in block order by the last block of that mesh to arrive (a
// per-mesh counter), which then takes the mesh's decision (CG step sizes and
// convergence, Newton tolerance and direction test, line-search acceptance)
// in device memory.  A whole timestep is one CUDA graph: three nested WHILE
// conditional nodes (Newton iterations, PCG iterations, line-search trials)
// whose conditions are set by one-block kernels from the per-mesh states, so
// the host launches one graph and reads the per-mesh statistics once.
//
// Launch shapes (lanes per row of the product, threads and rows per thread
// of the row kernels) are chosen by timing the candidates on the first
// timestep's assembled system (an autotuner); the graph is built for the
// winner.
#include "mls_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace mls {

enum { BPH_ASSEMBLE = 0, BPH_LS = 1, BPH_FINAL = 2, BPH_DONE = 3 };
enum { BC_PREP = 0, BC_SPMV, BC_UPD, BC_DIR, BC_ENERGY, BC_SMOOTH, BC_COUNT };

// per-mesh state (device)
struct BMesh {
  double g0, gnorm, E0, gd, alpha, step_rel;
  double bb, rr, rz, pq, alpha_p, beta, tol2;
  int phase, newton, pcg, trials, halvings, status, apply, start_bad;
  int iter, done, pad0, pad1;
};

struct BParams {        // per-timestep constants
  double h2, scale0, newton_tol, pcg_rtol, eta_floor;
  int max_newton, max_pcg;
  double kappa, dhat, po, pn0, pn1, pn2;
  int contact;
  double fmu, feps;       // lagged point-plane friction: coefficient (0: none), mollifier width
};

struct BView {
  int nmesh;
  // row blocks
  int nrb;
  const int* rb_mesh; const int* rb_row0; const int* rb_row1;
  const int* rb_first; const int* rb_count;
  // slices (32 rows)
  const int* sl_mesh; const int* sl_first; const int* sl_count;
  // tet blocks
  int ntb;
  const int* tb_mesh; const int* tb_t0; const int* tb_t1;
  const int* tb_first; const int* tb_count;
  const double* mass_min;        // [nmesh] smallest free-vertex mass
  unsigned* cnt;                 // [BC_COUNT][nmesh], left at zero
  double* part_rb;               // [nrb][4]
  double* part_sl;               // [n_slices]
  double* part_tb;               // [ntb][2]
  BMesh* M;
};

constexpr int kTetBlock = 256;

// ---- block reductions (any block size that is a multiple of 32, <= 1024) ----------------
template <int K>
__device__ __forceinline__ void bsum(double (&v)[K]) {
  __shared__ double sh[K][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    double s = v[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) sh[k][warp] = s;
  }
  __syncthreads();
  if (warp == 0) {
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

__device__ __forceinline__ double bmax(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    v = lane < nw ? sh[lane] : -1e300;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  __syncthreads();
  return v;
}

__device__ __forceinline__ double bmin(double v) { return -bmax(-v); }

// Arrival of this block for mesh m; true in the last block of the mesh to
// arrive (all its blocks' partials are then visible).  The counter is reset
// by that block.
__device__ __forceinline__ bool last_of_mesh(unsigned* counter, unsigned total) {
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(counter, 1u) == total - 1;
    if (last) *counter = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// ---- state kernels -----------------------------------------------------------------------
__global__ void k_breset(int nmesh, BMesh* __restrict__ M) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= nmesh) return;
  BMesh s{};
  s.phase = BPH_ASSEMBLE;
  s.status = MLS_OK;
  s.done = 1;
  s.alpha = 1.0;
  M[m] = s;
}

// user [n_user][3] -> internal padded [n][3]; dummy rows parked far from the plane
__global__ void k_bpack(int n, const int* __restrict__ vmap, const double* __restrict__ x,
                        const double* __restrict__ v, double* __restrict__ bx, double* __restrict__ bv,
                        double px, double py, double pz) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int u = vmap[i];
  if (u >= 0) {
#pragma unroll
    for (int k = 0; k < 3; ++k) { bx[3 * i + k] = x[3 * (int64_t)u + k]; bv[3 * i + k] = v[3 * (int64_t)u + k]; }
  } else {
    bx[3 * i] = px; bx[3 * i + 1] = py; bx[3 * i + 2] = pz;
    bv[3 * i] = 0.0; bv[3 * i + 1] = 0.0; bv[3 * i + 2] = 0.0;
  }
}

__global__ void k_bunpack(int n, const int* __restrict__ vmap, const Vec4d* __restrict__ xk,
                          const Vec4d* __restrict__ xt, double* __restrict__ dx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int u = vmap[i];
  if (u < 0) return;
  const Vec4d a = xk[i], b = xt[i];
  dx[3 * (int64_t)u] = a.x - b.x;
  dx[3 * (int64_t)u + 1] = a.y - b.y;
  dx[3 * (int64_t)u + 2] = a.z - b.z;
}

// ---- energy per mesh (tets, then vertices), three uses --------------------------------------
// MODE 0: at x^t (must be feasible); MODE 1: at the predictor (start there
// when feasible); MODE 2: a line-search trial x + alpha_m d.
struct BEnergyIn {
  int t;
  const int* tets; const double* Dminv; const double* vol; const double* mu; const double* lam;
  const double* mass; const uint8_t* pinned; const Vec4d* xtil;
  const Vec4d* xt;        // x^t, the friction lag state
};

template <int MODE>
__global__ void __launch_bounds__(kTetBlock) k_benergy(BView V, BEnergyIn in, BParams P, const Vec4d* __restrict__ x,
                                                       const Vec4d* __restrict__ d) {
  const bool tetblk = (int)blockIdx.x < V.ntb;
  const int b = tetblk ? blockIdx.x : blockIdx.x - V.ntb;
  const int m = tetblk ? V.tb_mesh[b] : V.rb_mesh[b];
  BMesh* M = V.M + m;
  const int phase = M->phase;
  if (MODE == 2 ? (phase != BPH_LS && phase != BPH_FINAL) : phase == BPH_DONE) return;
  const double alpha = MODE == 2 ? M->alpha : 0.0;
  double acc[2] = {0.0, 0.0};
  if (tetblk) {
    const int t = in.t;
    for (int e = V.tb_t0[b] + threadIdx.x; e < V.tb_t1[b]; e += blockDim.x) {
      Vec4d p[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int v = in.tets[a * t + e];
        Vec4d xv = x[v];
        if (MODE == 2) {
          const Vec4d dv = d[v];
          xv.x += alpha * dv.x; xv.y += alpha * dv.y; xv.z += alpha * dv.z;
        }
        p[a] = xv;
      }
      double F[3][3];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double e1 = a == 0 ? p[1].x - p[0].x : a == 1 ? p[1].y - p[0].y : p[1].z - p[0].z;
        const double e2 = a == 0 ? p[2].x - p[0].x : a == 1 ? p[2].y - p[0].y : p[2].z - p[0].z;
        const double e3 = a == 0 ? p[3].x - p[0].x : a == 1 ? p[3].y - p[0].y : p[3].z - p[0].z;
#pragma unroll
        for (int c = 0; c < 3; ++c)
          F[a][c] = e1 * in.Dminv[(0 + c) * t + e] + e2 * in.Dminv[(3 + c) * t + e] + e3 * in.Dminv[(6 + c) * t + e];
      }
      const double J = F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
                       F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
                       F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
      if (J > 0.0) {
        double I2 = 0.0;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int c = 0; c < 3; ++c) I2 += F[a][c] * F[a][c];
        const double lnJ = log(J), mu = in.mu[e], lam = in.lam[e];
        acc[0] += P.h2 * in.vol[e] * (0.5 * mu * (I2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
      } else {
        acc[1] += 1.0;
      }
    }
  } else {
    for (int v = V.rb_row0[b] + threadIdx.x; v < V.rb_row1[b]; v += blockDim.x) {
      Vec4d xv = x[v];
      if (MODE == 2) {
        const Vec4d dv = d[v];
        xv.x += alpha * dv.x; xv.y += alpha * dv.y; xv.z += alpha * dv.z;
      }
      if (!in.pinned[v]) {
        const Vec4d xt = in.xtil[v];
        const double ex = xv.x - xt.x, ey = xv.y - xt.y, ez = xv.z - xt.z;
        acc[0] += 0.5 * in.mass[v] * (ex * ex + ey * ey + ez * ez);
      }
      if (P.contact) {
        const double dist = P.pn0 * xv.x + P.pn1 * xv.y + P.pn2 * xv.z - P.po;
        if (dist <= 0.0) {
          acc[1] += 1.0;
        } else if (dist < P.dhat) {
          const double r = dist - P.dhat;
          acc[0] += P.h2 * P.kappa * (-r * r * log(dist / P.dhat));
        }
        if (P.fmu > 0.0) {
          // lagged friction mu lam f0(|slip|) (Eq. IP, term D), as in the single-mesh energy
          const Vec4d xtv = in.xt[v];
          const double lam = fric_lambda(P.pn0 * xtv.x + P.pn1 * xtv.y + P.pn2 * xtv.z - P.po, P.dhat, P.kappa);
          if (lam > 0.0) {
            double u[3];
            const double y = fric_slip(xv, xtv, P.pn0, P.pn1, P.pn2, u);
            acc[0] += P.h2 * P.fmu * lam * fric_f0(y, P.feps);
          }
        }
      }
    }
  }
  bsum<2>(acc);
  double* part = V.part_tb;  // tet blocks first, then row blocks, [ntb + nrb][2]
  if (threadIdx.x == 0) { part[2 * (int64_t)blockIdx.x] = acc[0]; part[2 * (int64_t)blockIdx.x + 1] = acc[1]; }
  const unsigned total = (unsigned)(V.tb_count[m] + V.rb_count[m]);
  if (!last_of_mesh(V.cnt + BC_ENERGY * V.nmesh + m, total)) return;
  double tot[2] = {0.0, 0.0};
  const int tb0 = V.tb_first[m], ntbm = V.tb_count[m], rb0 = V.rb_first[m], nrbm = V.rb_count[m];
  for (int i = threadIdx.x; i < ntbm + nrbm; i += blockDim.x) {
    const int64_t blk = i < ntbm ? (int64_t)(tb0 + i) : (int64_t)(V.ntb + rb0 + i - ntbm);
    tot[0] += __ldcg(part + 2 * blk);
    tot[1] += __ldcg(part + 2 * blk + 1);
  }
  bsum<2>(tot);
  if (threadIdx.x != 0) return;
  const double E = tot[0];
  const bool bad = tot[1] > 0.5 || !isfinite(E);
  if (MODE == 0) {
    if (bad) { M->status = MLS_EINVERTED; M->phase = BPH_DONE; }
    else M->E0 = E;
  } else if (MODE == 1) {
    M->start_bad = bad ? 1 : 0;
    if (!bad) M->E0 = E;
  } else {
    M->trials += 1;
    M->apply = 0;
    if (phase == BPH_FINAL) {
      // converged: the final (tiny) direction is applied in full when feasible
      M->apply = bad ? 0 : 1;
      if (!bad) M->E0 = E;
      M->phase = BPH_DONE;
      M->status = MLS_OK;
    } else {
      const double a = M->alpha, cgd = 1e-4 * a * M->gd;
      if (!bad && (fabs(cgd) <= 1e-13 * fabs(M->E0) || E <= M->E0 + cgd)) {
        M->apply = 1;
        M->E0 = E;
        M->phase = BPH_ASSEMBLE;
      } else {
        M->alpha = 0.5 * a;
        M->halvings += 1;
        if (M->halvings > 60) { M->status = MLS_ELINESEARCH; M->phase = BPH_DONE; }
      }
    }
  }
}

// meshes whose predictor is infeasible start from x^t
__global__ void k_bselect(BView V, const Vec4d* __restrict__ xt, Vec4d* __restrict__ xk) {
  const int m = V.rb_mesh[blockIdx.x];
  if (!V.M[m].start_bad) return;
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) xk[v] = xt[v];
}

// x += alpha d for meshes whose trial was accepted
__global__ void k_bapply(BView V, Vec4d* __restrict__ xk, const Vec4d* __restrict__ d) {
  const int m = V.rb_mesh[blockIdx.x];
  const BMesh* M = V.M + m;
  if (!M->apply) return;
  const double a = M->alpha;
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) {
    Vec4d xv = xk[v];
    const Vec4d dv = d[v];
    xv.x += a * dv.x; xv.y += a * dv.y; xv.z += a * dv.z;
    xk[v] = xv;
  }
}

// ---- Newton iteration start: PCG initialisation and tolerance per mesh ---------------------
// two_level: z receives the smoothing term omega D^{-1} b of the first cycle
// (r.z then comes from the cycle's post-smoothing); otherwise z = D^{-1} b
// and r.z are formed here.
template <typename VT>
__global__ void k_bprep(BView V, BParams P, int two_level, VT omega, const Vec4d* __restrict__ grad,
                        const Vec4<VT>* __restrict__ b, const VT* __restrict__ dinv, const Vec4d* __restrict__ xk,
                        const Vec4d* __restrict__ xt, Vec4<VT>* __restrict__ x, Vec4<VT>* __restrict__ r,
                        Vec4<VT>* __restrict__ z, Vec4<VT>* __restrict__ p, Vec4<VT>* __restrict__ q) {
  const int m = V.rb_mesh[blockIdx.x];
  BMesh* M = V.M + m;
  if (M->phase != BPH_ASSEMBLE) return;
  double acc[2] = {0.0, 0.0};  // g.g, r.z
  double xd = 0.0;
  const Vec4<VT> zero{VT(0), VT(0), VT(0), VT(0)};
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) {
    const Vec4d g = grad[v];
    acc[0] += g.x * g.x + g.y * g.y + g.z * g.z;
    const Vec4<VT> bv = b[v];
    const VT* D = dinv + (int64_t)v * 9;
    const VT w = two_level ? omega : VT(1);
    const Vec4<VT> zv{w * (D[0] * bv.x + D[1] * bv.y + D[2] * bv.z), w * (D[3] * bv.x + D[4] * bv.y + D[5] * bv.z),
                      w * (D[6] * bv.x + D[7] * bv.y + D[8] * bv.z), VT(0)};
    x[v] = zero; p[v] = zero; q[v] = zero;
    r[v] = bv;
    z[v] = zv;
    if (!two_level) acc[1] += (double)bv.x * zv.x + (double)bv.y * zv.y + (double)bv.z * zv.z;
    const Vec4d a = xk[v], c = xt[v];
    xd = fmax(xd, fmax(fabs(a.x - c.x), fmax(fabs(a.y - c.y), fabs(a.z - c.z))));
  }
  bsum<2>(acc);
  xd = bmax(xd);
  double* part = V.part_rb + 4 * (int64_t)blockIdx.x;
  if (threadIdx.x == 0) { part[0] = acc[0]; part[1] = acc[1]; part[2] = xd; }
  if (!last_of_mesh(V.cnt + BC_PREP * V.nmesh + m, (unsigned)V.rb_count[m])) return;
  double tot[2] = {0.0, 0.0};
  double xdm = 0.0;
  const int rb0 = V.rb_first[m], nrbm = V.rb_count[m];
  for (int i = threadIdx.x; i < nrbm; i += blockDim.x) {
    const double* pp = V.part_rb + 4 * (int64_t)(rb0 + i);
    tot[0] += __ldcg(pp);
    tot[1] += __ldcg(pp + 1);
    xdm = fmax(xdm, __ldcg(pp + 2));
  }
  bsum<2>(tot);
  xdm = bmax(xdm);
  if (threadIdx.x != 0) return;
  M->newton += 1;
  const double gnorm = sqrt(tot[0]);
  M->gnorm = gnorm;
  if (M->newton == 1) M->g0 = gnorm;
  M->iter = 0;
  M->beta = 0.0;
  if (!isfinite(gnorm)) { M->status = MLS_ENONFINITE; M->phase = BPH_DONE; M->done = 1; return; }
  if (gnorm == 0.0) { M->step_rel = 0.0; M->status = MLS_OK; M->phase = BPH_DONE; M->done = 1; return; }
  // forcing term: min(rtol, sqrt(|g| / |g0|)), floored; absolute floor from
  // H >= M: a residual below 0.01 tol scale m_min cannot move the step test
  double eta = fmin(P.pcg_rtol, sqrt(gnorm / M->g0));
  eta = fmax(eta, P.eta_floor);
  const double abs_floor = 0.01 * P.newton_tol * fmax(xdm, P.scale0) * V.mass_min[m];
  eta = fmax(eta, abs_floor / gnorm);
  M->bb = tot[0];
  M->rr = tot[0];
  M->rz = tot[1];
  M->tol2 = eta * eta * tot[0];
  M->done = 0;
}

// ---- PCG iteration (block Jacobi), per-mesh scalars ---------------------------------------
// Product: one slice (32 rows) per block, LANES lanes per row (4 or 8).
template <typename VT, typename MT, int LANES>
__global__ void __launch_bounds__(32 * LANES) k_bspmv(BView V, int n, const int* __restrict__ slice_ptr,
                                                      const int* __restrict__ col, const int* __restrict__ row_len,
                                                      const MT* __restrict__ val, const Vec4<VT>* __restrict__ z,
                                                      Vec4<VT>* __restrict__ p, Vec4<VT>* __restrict__ q) {
  chain_wait();
  chain_release();
  const int s = blockIdx.x;
  const int m = V.sl_mesh[s];
  BMesh* M = V.M + m;
  if (M->phase != BPH_ASSEMBLE || M->done) return;
  const int part = threadIdx.x % LANES, rl = threadIdx.x / LANES;
  const int row = s * 32 + rl;
  const int len = row < n ? row_len[row] : 0;
  const int64_t g0 = slice_ptr[s];
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
  constexpr int U = 16 / LANES;
  for (int k0 = part; k0 < len; k0 += 16) {
    int c[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int k = k0 + LANES * u;
      ok[u] = k < len;
      c[u] = ok[u] ? __ldg(col + (g0 + k) * 32 + rl) : 0;
    }
    Vec4<VT> xv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) xv[u] = ok[u] ? z[c[u]] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const MT* v = val + (g0 + k0 + LANES * u) * 288 + rl;
      y0 += load_as<VT>(v[0]) * xv[u].x + load_as<VT>(v[32]) * xv[u].y + load_as<VT>(v[64]) * xv[u].z;
      y1 += load_as<VT>(v[96]) * xv[u].x + load_as<VT>(v[128]) * xv[u].y + load_as<VT>(v[160]) * xv[u].z;
      y2 += load_as<VT>(v[192]) * xv[u].x + load_as<VT>(v[224]) * xv[u].y + load_as<VT>(v[256]) * xv[u].z;
    }
  }
#pragma unroll
  for (int o = 1; o < LANES; o <<= 1) {
    y0 += __shfl_xor_sync(0xffffffffu, y0, o);
    y1 += __shfl_xor_sync(0xffffffffu, y1, o);
    y2 += __shfl_xor_sync(0xffffffffu, y2, o);
  }
  double acc[1] = {0.0};
  if (part == 0 && row < n) {
    const VT beta = (VT)M->beta;
    const Vec4<VT> zv = z[row], pv = p[row], qv = q[row];
    const Vec4<VT> pn{zv.x + beta * pv.x, zv.y + beta * pv.y, zv.z + beta * pv.z, VT(0)};
    const Vec4<VT> qn{y0 + beta * qv.x, y1 + beta * qv.y, y2 + beta * qv.z, VT(0)};
    p[row] = pn;
    q[row] = qn;
    acc[0] = (double)pn.x * qn.x + (double)pn.y * qn.y + (double)pn.z * qn.z;
  }
  bsum<1>(acc);
  if (threadIdx.x == 0) V.part_sl[s] = acc[0];
  if (!last_of_mesh(V.cnt + BC_SPMV * V.nmesh + m, (unsigned)V.sl_count[m])) return;
  double tot[1] = {0.0};
  const int s0 = V.sl_first[m], nsm = V.sl_count[m];
  for (int i = threadIdx.x; i < nsm; i += blockDim.x) tot[0] += __ldcg(V.part_sl + s0 + i);
  bsum<1>(tot);
  if (threadIdx.x != 0) return;
  M->pq = tot[0];
  if (tot[0] > 0.0 && isfinite(tot[0])) {
    M->alpha_p = M->rz / tot[0];
  } else {
    M->alpha_p = 0.0;
    M->done = 3;  // breakdown: H or the preconditioner is not positive definite
  }
}

// two_level: z = omega D^{-1} r (the cycle's pre-smoothing; r.z and beta
// come from its post-smoothing); otherwise z = D^{-1} r with r.z and beta
template <typename VT>
__global__ void k_bupdate(BView V, int max_iter, int two_level, VT omega, const VT* __restrict__ dinv,
                          Vec4<VT>* __restrict__ x, Vec4<VT>* __restrict__ r, Vec4<VT>* __restrict__ z,
                          const Vec4<VT>* __restrict__ p, const Vec4<VT>* __restrict__ q) {
  chain_wait();
  chain_release();
  const int m = V.rb_mesh[blockIdx.x];
  BMesh* M = V.M + m;
  if (M->phase != BPH_ASSEMBLE || M->done) return;
  const VT alpha = (VT)M->alpha_p;
  double acc[2] = {0.0, 0.0};  // r.r, r.z
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) {
    const Vec4<VT> pv = p[v], qv = q[v];
    Vec4<VT> xv = x[v], rv = r[v];
    xv.x += alpha * pv.x; xv.y += alpha * pv.y; xv.z += alpha * pv.z;
    rv.x -= alpha * qv.x; rv.y -= alpha * qv.y; rv.z -= alpha * qv.z;
    x[v] = xv;
    r[v] = rv;
    const VT* D = dinv + (int64_t)v * 9;
    const VT w = two_level ? omega : VT(1);
    const Vec4<VT> zv{w * (D[0] * rv.x + D[1] * rv.y + D[2] * rv.z), w * (D[3] * rv.x + D[4] * rv.y + D[5] * rv.z),
                      w * (D[6] * rv.x + D[7] * rv.y + D[8] * rv.z), VT(0)};
    z[v] = zv;
    acc[0] += (double)rv.x * rv.x + (double)rv.y * rv.y + (double)rv.z * rv.z;
    acc[1] += (double)rv.x * zv.x + (double)rv.y * zv.y + (double)rv.z * zv.z;
  }
  bsum<2>(acc);
  double* part = V.part_rb + 4 * (int64_t)blockIdx.x;
  if (threadIdx.x == 0) { part[0] = acc[0]; part[1] = acc[1]; }
  if (!last_of_mesh(V.cnt + BC_UPD * V.nmesh + m, (unsigned)V.rb_count[m])) return;
  double tot[2] = {0.0, 0.0};
  const int rb0 = V.rb_first[m], nrbm = V.rb_count[m];
  for (int i = threadIdx.x; i < nrbm; i += blockDim.x) {
    tot[0] += __ldcg(V.part_rb + 4 * (int64_t)(rb0 + i));
    tot[1] += __ldcg(V.part_rb + 4 * (int64_t)(rb0 + i) + 1);
  }
  bsum<2>(tot);
  if (threadIdx.x != 0) return;
  M->rr = tot[0];
  M->iter += 1;
  if (!isfinite(tot[0])) { M->done = 3; return; }
  if (tot[0] <= M->tol2) { M->done = 1; return; }
  if (M->iter >= max_iter) { M->done = 2; return; }
  if (two_level) return;
  M->beta = tot[1] / M->rz;
  M->rz = tot[1];
}

// ---- direction: step test, descent test, CCD bound -----------------------------------------
template <typename VT>
__global__ void k_bdir(BView V, BParams P, const Vec4<VT>* __restrict__ xs, const uint8_t* __restrict__ pinned,
                       const Vec4d* __restrict__ grad, const Vec4d* __restrict__ xk, const Vec4d* __restrict__ xt,
                       Vec4d* __restrict__ d) {
  const int m = V.rb_mesh[blockIdx.x];
  BMesh* M = V.M + m;
  if (M->phase != BPH_ASSEMBLE) return;
  double dinf = 0.0, xd = 0.0, tmin = 1e300;
  double acc[1] = {0.0};
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) {
    Vec4d dv{0.0, 0.0, 0.0, 0.0};
    if (!pinned[v]) {
      const Vec4<VT> s = xs[v];
      dv = Vec4d{(double)s.x, (double)s.y, (double)s.z, 0.0};
    }
    d[v] = dv;
    dinf = fmax(dinf, fmax(fabs(dv.x), fmax(fabs(dv.y), fabs(dv.z))));
    const Vec4d a = xk[v], c = xt[v];
    xd = fmax(xd, fmax(fabs(a.x - c.x), fmax(fabs(a.y - c.y), fabs(a.z - c.z))));
    const Vec4d g = grad[v];
    acc[0] += g.x * dv.x + g.y * dv.y + g.z * dv.z;
    if (P.contact && !pinned[v]) {
      const double nd = P.pn0 * dv.x + P.pn1 * dv.y + P.pn2 * dv.z;
      if (nd < 0.0) {
        const double dist = P.pn0 * a.x + P.pn1 * a.y + P.pn2 * a.z - P.po;
        tmin = fmin(tmin, fmax(dist, 0.0) / (-nd));
      }
    }
  }
  bsum<1>(acc);
  dinf = bmax(dinf);
  xd = bmax(xd);
  tmin = bmin(tmin);
  double* part = V.part_rb + 4 * (int64_t)blockIdx.x;
  if (threadIdx.x == 0) { part[0] = acc[0]; part[1] = dinf; part[2] = xd; part[3] = tmin; }
  if (!last_of_mesh(V.cnt + BC_DIR * V.nmesh + m, (unsigned)V.rb_count[m])) return;
  double tot[1] = {0.0};
  double dm = 0.0, xm = 0.0, tm = 1e300;
  const int rb0 = V.rb_first[m], nrbm = V.rb_count[m];
  for (int i = threadIdx.x; i < nrbm; i += blockDim.x) {
    const double* pp = V.part_rb + 4 * (int64_t)(rb0 + i);
    tot[0] += __ldcg(pp);
    dm = fmax(dm, __ldcg(pp + 1));
    xm = fmax(xm, __ldcg(pp + 2));
    tm = fmin(tm, __ldcg(pp + 3));
  }
  bsum<1>(tot);
  dm = bmax(dm);
  xm = bmax(xm);
  tm = bmin(tm);
  if (threadIdx.x != 0) return;
  M->pcg += M->iter;
  const int pcg_state = M->done;
  M->done = 1;
  // a breakdown of the solve (non-positive curvature or a non-finite value)
  // fails the mesh's step, as in the single-mesh timestep
  if (pcg_state == 3 || !isfinite(dm) || !isfinite(tot[0])) { M->status = MLS_ENONFINITE; M->phase = BPH_DONE; return; }
  const double step_rel = dm / fmax(xm, P.scale0);
  M->step_rel = step_rel;
  M->gd = tot[0];
  M->halvings = 0;
  if (step_rel <= P.newton_tol) {
    M->alpha = 1.0;
    M->phase = BPH_FINAL;
    return;
  }
  if (!(tot[0] < 0.0)) { M->status = MLS_ELINESEARCH; M->phase = BPH_DONE; return; }
  M->alpha = (P.contact && tm < 1e299) ? fmin(1.0, 0.9 * tm) : 1.0;
  M->phase = BPH_LS;
}

// ---- loop conditions (one block) ---------------------------------------------------------
// which: 0 PCG (some mesh still iterating), 1 line search (some mesh still
// searching; clears the accept flags), 2 Newton (some mesh not done; caps
// the iteration count).  *trip counts the evaluations.
// trip_cap bounds the evaluations of one loop condition per timestep (the
// largest count the per-mesh iteration caps allow): should it ever be
// reached, the loop ends and the meshes still in it are marked not converged,
// so a graph loop cannot run without end.
__global__ void k_bcond(int nmesh, BMesh* __restrict__ M, int which, int max_newton, cudaGraphConditionalHandle h,
                        int use_handle, int* __restrict__ any_out, int* __restrict__ trip, int trip_cap) {
  __shared__ int any;
  if (threadIdx.x == 0) any = 0;
  __syncthreads();
  const bool capped = *trip >= trip_cap;
  int mine = 0;
  for (int m = threadIdx.x; m < nmesh; m += blockDim.x) {
    BMesh* s = M + m;
    if (which == 0) {
      mine |= (s->phase == BPH_ASSEMBLE && !s->done) ? 1 : 0;
    } else if (which == 1) {
      s->apply = 0;
      mine |= (s->phase == BPH_LS || s->phase == BPH_FINAL) ? 1 : 0;
    } else {
      if (s->phase == BPH_ASSEMBLE && s->newton >= max_newton) {
        s->status = MLS_ENOTCONV;
        s->phase = BPH_DONE;
      }
      mine |= s->phase != BPH_DONE ? 1 : 0;
    }
  }
  if (mine) atomicOr(&any, 1);
  __syncthreads();
  if (capped && any) {
    for (int m = threadIdx.x; m < nmesh; m += blockDim.x) {
      BMesh* s = M + m;
      if (s->phase != BPH_DONE) {
        s->status = MLS_ENOTCONV;
        s->phase = BPH_DONE;
        s->done = 1;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) any = 0;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (use_handle) cudaGraphSetConditional(h, any ? 1u : 0u);
    if (any_out) *any_out = any;
    *trip += 1;
  }
}


// ---- two-level preconditioning per mesh --------------------------------------------------
// Each mesh has its own SMS basis (handles numbered globally, a mesh's
// handles contiguous); U is block diagonal, so U^T H U is block diagonal too
// and the dense Galerkin product leaves only each mesh's diagonal block
// non-zero.  Each block is factored in float64 by one CTA (right-looking
// Cholesky), its inverse factor W_m = L_m^{-1} formed column by column, and
// the coarse solve is W_m^T (W_m c_m) per mesh.
constexpr int kMaxCoarseRows = 1536;   // 128 handles per mesh

struct BCoarse {
  int r;                   // total coarse rows (12 x handles)
  const int* coff;         // [nmesh] first coarse row of each mesh
  const int* csz;          // [nmesh] coarse rows of each mesh
  const int64_t* woff;     // [nmesh] first entry of the mesh's W block (csz^2 entries)
  const int* crow_mesh;    // [r] mesh of each coarse row
  const int* hmesh;        // [m] mesh of each handle
};

__device__ __forceinline__ bool pcg_active(const BMesh* M) { return M->phase == BPH_ASSEMBLE && !M->done; }

// right-looking Cholesky of the mesh's diagonal block of A (float64, leading
// dimension ld), in place.  The block's lower triangle is saved to the same
// place in S first; a non-positive pivot restores it with the diagonal
// scaled by 1 + sigma and factors again (kShiftTries retries, sigma from
// kShiftFirst growing kShiftGrowth-fold); if the last retry fails too, the
// mesh fails (MLS_ECHOL)
__global__ void __launch_bounds__(256) k_bchol(BView V, BCoarse C, double* __restrict__ A, double* __restrict__ S,
                                               int ld) {
  const int m = blockIdx.x;
  BMesh* M = V.M + m;
  if (M->phase == BPH_DONE) return;
  const int o = C.coff[m], n = C.csz[m];
  double* a = A + (int64_t)o * ld + o;
  double* sv = S + (int64_t)o * ld + o;
  __shared__ double col[kMaxCoarseRows];
  __shared__ int bad;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw)
    for (int k = lane; k <= i; k += 32) sv[(int64_t)i * ld + k] = a[(int64_t)i * ld + k];
  double sigma = 0.0;
  for (int attempt = 0; attempt <= kShiftTries; ++attempt) {
    if (attempt > 0) {
      sigma = attempt == 1 ? kShiftFirst : sigma * kShiftGrowth;
      __syncthreads();
      for (int i = warp; i < n; i += nw)
        for (int k = lane; k <= i; k += 32) {
          const double s0 = sv[(int64_t)i * ld + k];
          a[(int64_t)i * ld + k] = (k == i) ? s0 + sigma * fmax(s0, 0.0) : s0;
        }
    }
    if (threadIdx.x == 0) bad = 0;
    for (int j = 0; j < n; ++j) {
      __syncthreads();
      const double d = a[(int64_t)j * ld + j];
      if (!(d > 0.0) || !isfinite(d)) {
        if (threadIdx.x == 0) bad = j + 1;
        break;
      }
      const double piv = sqrt(d), inv = 1.0 / piv;
      for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
        const double v = a[(int64_t)i * ld + j] * inv;
        a[(int64_t)i * ld + j] = v;
        col[i] = v;
      }
      __syncthreads();
      if (threadIdx.x == 0) a[(int64_t)j * ld + j] = piv;
      for (int i = j + 1 + warp; i < n; i += nw) {
        const double li = col[i];
        double* ai = a + (int64_t)i * ld;
        for (int k = j + 1 + lane; k <= i; k += 32) ai[k] -= li * col[k];
      }
    }
    __syncthreads();
    if (!bad) break;
  }
  if (threadIdx.x == 0 && bad) {
    M->status = MLS_ECHOL;
    M->phase = BPH_DONE;
    M->done = 1;
  }
}

// W_m = L_m^{-1} (lower triangular) by forward substitution, one column per
// thread, in float64 (scratch S, same layout as A), stored in solve
// precision in W; then the dense block inverse A_m^{-1} = W_m^T W_m into WT
// (row-major csz x csz blocks at woff)
template <typename VT>
__global__ void __launch_bounds__(256) k_btrinv(BView V, BCoarse C, const double* __restrict__ A,
                                                double* __restrict__ S, int ld, VT* __restrict__ W,
                                                VT* __restrict__ WT) {
  const int m = blockIdx.x;
  if (V.M[m].phase == BPH_DONE) return;
  const int o = C.coff[m], n = C.csz[m];
  const double* L = A + (int64_t)o * ld + o;
  double* w = S + (int64_t)o * ld + o;
  VT* Wm = W + C.woff[m];
  VT* WTm = WT + C.woff[m];
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    for (int i = 0; i < n; ++i) {
      double v = 0.0;
      if (i == c) {
        v = 1.0 / L[(int64_t)i * ld + i];
      } else if (i > c) {
        double acc = 0.0;
        const double* Li = L + (int64_t)i * ld;
        for (int k = c; k < i; ++k) acc += Li[k] * w[(int64_t)k * ld + c];
        v = -acc / Li[i];
      }
      w[(int64_t)i * ld + c] = v;
      Wm[(int64_t)i * n + c] = (VT)v;
    }
  }
  __syncthreads();
  // the block's dense inverse A_m^{-1} = W_m^T W_m (solve precision, into WT):
  // entry (i, j), j <= i, sums W[k][i] W[k][j] over k >= i; mirrored
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    if (j > i) continue;
    VT acc = VT(0);
    for (int k = i; k < n; ++k) acc += Wm[(int64_t)k * n + i] * Wm[(int64_t)k * n + j];
    WTm[(int64_t)i * n + j] = acc;
    WTm[(int64_t)j * n + i] = acc;
  }
}

// y = W x (lower = 1), W^T x (lower = 0) or, lower = 2, the dense block
// product per mesh; four warps per coarse row, 16-byte loads
template <typename VT>
__global__ void __launch_bounds__(256) k_btrigemv(BView V, BCoarse C, const VT* __restrict__ W, int lower,
                                                  const VT* __restrict__ x, VT* __restrict__ y) {
  chain_wait();
  chain_release();
  constexpr int EV = 16 / sizeof(VT);
  constexpr int WPR = 4;
  __shared__ VT part[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = blockIdx.x * (8 / WPR) + warp / WPR;
  const int sub = warp % WPR;
  VT acc = VT(0);
  bool on = false;
  if (g < C.r) {
    const int m = C.crow_mesh[g];
    on = pcg_active(V.M + m);
    if (on) {
      const int o = C.coff[m], n = C.csz[m], i = g - o;
      const int v0 = lower ? 0 : i / EV;
      const int v1 = lower == 1 ? (i + EV) / EV : n / EV;
      using V16 = typename std::conditional<sizeof(VT) == 4, float4, double2>::type;
      const V16* Wr = reinterpret_cast<const V16*>(W + C.woff[m] + (int64_t)i * n);
      const V16* xv = reinterpret_cast<const V16*>(x + o);
      for (int c = v0 + sub * 32 + lane; c < v1; c += 32 * WPR) {
        const V16 a = Wr[c];
        const V16 b = xv[c];
        if constexpr (sizeof(VT) == 4) acc += a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w;
        else acc += a.x * b.x + a.y * b.y;
      }
    }
  }
#pragma unroll
  for (int o2 = 16; o2 > 0; o2 >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o2);
  if (lane == 0) part[warp] = acc;
  __syncthreads();
  if (on && sub == 0 && lane == 0) {
    VT t = VT(0);
#pragma unroll
    for (int k = 0; k < WPR; ++k) t += part[warp + k];
    y[g] = t;
  }
}

// c_j = sum_{v in supp j} phi_j(v) t_v (x) a_vj, one warp per chunk of a
// handle's entries (as the single-mesh restriction), meshes done skipped
struct BBasisView {
  const void* vcoef; const void* hcoef;
  const int* vrow; const int* vh; const int* hrow; const int* hv;
  const int* rchunk_handle; const int* rchunk_beg; const int* rchunk_ptr;
  double* rpart; unsigned* rcount; int nrchunk;
};
constexpr int kBRestrictChunk = 256;

template <typename VT>
__global__ void __launch_bounds__(256) k_brestrict(BView V, BCoarse C, BBasisView B, const Vec4<VT>* __restrict__ t,
                                                   VT* __restrict__ c) {
  chain_wait();
  chain_release();
  const int lane = threadIdx.x & 31;
  const int ch = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (ch >= B.nrchunk) return;
  const int j = B.rchunk_handle[ch];
  if (!pcg_active(V.M + C.hmesh[j])) return;
  const int p0 = B.rchunk_beg[ch];
  const int p1 = min(p0 + kBRestrictChunk, B.hrow[j + 1]);
  constexpr int U = kBRestrictChunk / 32;
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
    const Vec4<VT> rv = t[hv[u]];
    const VT rc[3] = {rv.x, rv.y, rv.z};
    const VT av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
    for (int cc = 0; cc < 3; ++cc)
#pragma unroll
      for (int l = 0; l < 4; ++l) acc[4 * cc + l] += rc[cc] * av[l];
  }
#pragma unroll
  for (int q = 0; q < 12; ++q)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
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
    const double s = ordered_sum_ldcg(B.rpart + lane, 12, B.rchunk_ptr[j], B.rchunk_ptr[j + 1]);
    c[12 * (int64_t)j + lane] = (VT)s;
  }
  if (lane == 0) B.rcount[j] = 0;
}

// z1 += U c over the rows of active meshes
template <typename VT>
__global__ void k_bprolong(BView V, BBasisView B, const VT* __restrict__ c, Vec4<VT>* __restrict__ z1) {
  chain_wait();
  chain_release();
  const int m = V.rb_mesh[blockIdx.x];
  if (!pcg_active(V.M + m)) return;
  const Vec4<VT>* coef = (const Vec4<VT>*)B.vcoef;
  for (int v = V.rb_row0[blockIdx.x] + threadIdx.x; v < V.rb_row1[blockIdx.x]; v += blockDim.x) {
    VT o0 = VT(0), o1 = VT(0), o2 = VT(0);
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
        const Vec4<VT>* qj = (const Vec4<VT>*)(c + 12 * (int64_t)h[u]);
        const Vec4<VT> q0 = qj[0], q1 = qj[1], q2 = qj[2];
        o0 += a[u].x * q0.x + a[u].y * q0.y + a[u].z * q0.z + a[u].w * q0.w;
        o1 += a[u].x * q1.x + a[u].y * q1.y + a[u].z * q1.z + a[u].w * q1.w;
        o2 += a[u].x * q2.x + a[u].y * q2.y + a[u].z * q2.z + a[u].w * q2.w;
      }
    }
    const Vec4<VT> zb = z1[v];
    z1[v] = Vec4<VT>{zb.x + o0, zb.y + o1, zb.z + o2, VT(0)};
  }
}

// product of one slice of H with z (four lanes per row); rows of the slice
// returned in y of the lane with part == 0
template <typename VT, typename MT>
__device__ __forceinline__ void bslice_product(int n, const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                               const int* __restrict__ row_len, const MT* __restrict__ val, int s,
                                               const Vec4<VT>* __restrict__ z, VT (&y)[3]) {
  const int part = threadIdx.x & 3, rl = threadIdx.x >> 2;
  const int row = s * 32 + rl;
  const int len = row < n ? row_len[row] : 0;
  const int64_t g0 = slice_ptr[s];
  VT y0 = VT(0), y1 = VT(0), y2 = VT(0);
  for (int k0 = part; k0 < len; k0 += 16) {
    int cc[4];
    bool ok[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int k = k0 + 4 * u;
      ok[u] = k < len;
      cc[u] = ok[u] ? __ldg(col + (g0 + k) * 32 + rl) : 0;
    }
    Vec4<VT> xv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) xv[u] = ok[u] ? z[cc[u]] : Vec4<VT>{VT(0), VT(0), VT(0), VT(0)};
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

// t = r - H z1 (the residual of the pre-smoothed iterate), active meshes
template <typename VT, typename MT>
__global__ void __launch_bounds__(128) k_bresidual(BView V, int n, const int* __restrict__ slice_ptr,
                                                   const int* __restrict__ col, const int* __restrict__ row_len,
                                                   const MT* __restrict__ val, const Vec4<VT>* __restrict__ r,
                                                   const Vec4<VT>* __restrict__ z1, Vec4<VT>* __restrict__ t) {
  chain_wait();
  chain_release();
  const int s = blockIdx.x;
  if (!pcg_active(V.M + V.sl_mesh[s])) return;
  VT y[3];
  bslice_product<VT, MT>(n, slice_ptr, col, row_len, val, s, z1, y);
  const int row = s * 32 + (threadIdx.x >> 2);
  if ((threadIdx.x & 3) == 0 && row < n) {
    const Vec4<VT> rv = r[row];
    t[row] = Vec4<VT>{rv.x - y[0], rv.y - y[1], rv.z - y[2], VT(0)};
  }
}

// zf = z1 + omega D^{-1} (r - H z1) and r.zf per mesh (beta = 0 when first)
template <typename VT, typename MT>
__global__ void __launch_bounds__(128) k_bpost_smooth(BView V, int first, VT omega, int n,
                                                      const int* __restrict__ slice_ptr, const int* __restrict__ col,
                                                      const int* __restrict__ row_len, const MT* __restrict__ val,
                                                      const VT* __restrict__ dinv, const Vec4<VT>* __restrict__ r,
                                                      const Vec4<VT>* __restrict__ z1, Vec4<VT>* __restrict__ zf) {
  chain_wait();
  chain_release();
  const int s = blockIdx.x;
  const int m = V.sl_mesh[s];
  BMesh* M = V.M + m;
  if (!pcg_active(M)) return;
  VT y[3];
  bslice_product<VT, MT>(n, slice_ptr, col, row_len, val, s, z1, y);
  const int row = s * 32 + (threadIdx.x >> 2);
  double acc[1] = {0.0};
  if ((threadIdx.x & 3) == 0 && row < n) {
    const Vec4<VT> rv = r[row], zv = z1[row];
    const VT t0 = rv.x - y[0], t1 = rv.y - y[1], t2 = rv.z - y[2];
    const VT* D = dinv + (int64_t)row * 9;
    const Vec4<VT> zo{zv.x + omega * (D[0] * t0 + D[1] * t1 + D[2] * t2),
                      zv.y + omega * (D[3] * t0 + D[4] * t1 + D[5] * t2),
                      zv.z + omega * (D[6] * t0 + D[7] * t1 + D[8] * t2), VT(0)};
    zf[row] = zo;
    acc[0] = (double)rv.x * zo.x + (double)rv.y * zo.y + (double)rv.z * zo.z;
  }
  bsum<1>(acc);
  if (threadIdx.x == 0) V.part_sl[s] = acc[0];
  if (!last_of_mesh(V.cnt + BC_SMOOTH * V.nmesh + m, (unsigned)V.sl_count[m])) return;
  double tot[1] = {0.0};
  const int s0 = V.sl_first[m], nsm = V.sl_count[m];
  for (int i = threadIdx.x; i < nsm; i += blockDim.x) tot[0] += __ldcg(V.part_sl + s0 + i);
  bsum<1>(tot);
  if (threadIdx.x != 0) return;
  M->beta = first ? 0.0 : tot[0] / M->rz;
  M->rz = tot[0];
  if (!(tot[0] > 0.0) || !isfinite(tot[0])) M->done = (M->rr <= M->tol2) ? 1 : 3;
}

}  // namespace mls

using namespace mls;

// ---- the batch object ----------------------------------------------------------------------
struct BShape {
  int lanes = 4;        // lanes per row of the product (4 or 8)
  int row_threads = 256;
  int rows_per_thread = 1;
};

struct mls_batch {
  mls_ctx* ctx = nullptr;
  std::string err;
  int nmesh = 0;
  int n_user = 0;       // concatenated user vertices
  int n = 0;            // padded internal vertices
  std::vector<int> h_voff, h_toff, h_ioff, h_ipad;   // user vertex offsets, tet offsets, internal offsets, padded sizes
  std::vector<int> h_vmap;
  int* vmap = nullptr;  // [n] internal -> user vertex (-1: dummy)
  double* bx = nullptr; // [n][3] packed x, v
  double* bv = nullptr;
  double* bxp = nullptr; // [n][3] packed x^{t-1}, v^{t-1} (BDF2 steps; allocated on the first one)
  double* bvp = nullptr;
  bool bdf2 = false;     // the current step integrates with BDF2
  BMesh* M = nullptr;
  BMesh* h_M = nullptr; // pinned
  int* trips = nullptr; // [3] device
  int* h_trips = nullptr;
  int* any = nullptr;
  double* mass_min = nullptr;
  unsigned* cnt = nullptr;
  double* part_rb = nullptr;
  double* part_sl = nullptr;
  double* part_e = nullptr;
  // tables of the current shape
  BShape shape;
  bool tuned = false;
  double tune_ms = 0.0;
  std::vector<void*> tables;   // device allocations of the current tables
  BView view{};
  int nrb = 0, ntb = 0;
  // graph
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  double graph_dt = -1.0;
  bool graph_bdf2 = false;  // the integrator the graph was captured for
  bool graph_dirty = true;
  int64_t launches_fixed = 0, launches_newton = 0, launches_pcg = 0, launches_ls = 0;
  // two-level preconditioning (per-mesh bases)
  bool two_level = false;
  bool has_basis = false;
  BCoarse coarse{};
  std::vector<void*> coarse_alloc;
  void* W = nullptr;      // block-diagonal inverse factors, solve precision
  void* WT = nullptr;
  bool galerkin_warm = false;
};

namespace {

mls_status bfail(mls_batch* b, mls_status st, const std::string& msg) {
  b->err = msg;
  return st;
}

mls_status bcheck(mls_batch* b, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return MLS_OK;
  cudaGetLastError();
  return bfail(b, MLS_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

template <typename T>
mls_status bupload(mls_batch* b, std::vector<void*>& list, T** dst, const std::vector<T>& src) {
  void* p = nullptr;
  const size_t bytes = sizeof(T) * std::max<size_t>(src.size(), 1);
  if (cudaMalloc(&p, bytes) != cudaSuccess) { cudaGetLastError(); return bfail(b, MLS_ENOMEM, "batch table allocation"); }
  list.push_back(p);
  *dst = (T*)p;
  if (!src.empty()) return bcheck(b, cudaMemcpy(p, src.data(), sizeof(T) * src.size(), cudaMemcpyHostToDevice), "table upload");
  return MLS_OK;
}

void free_tables(mls_batch* b) {
  for (void* p : b->tables) cudaFree(p);
  b->tables.clear();
}

// row blocks, slices and tet blocks for one launch shape
mls_status build_tables(mls_batch* b, const BShape& sh) {
  free_tables(b);
  const int B = b->nmesh;
  const int rows_per_block = sh.row_threads * sh.rows_per_thread;
  std::vector<int> rb_mesh, rb_row0, rb_row1, rb_first(B), rb_count(B);
  std::vector<int> sl_mesh(b->n / 32), sl_first(B), sl_count(B);
  std::vector<int> tb_mesh, tb_t0, tb_t1, tb_first(B), tb_count(B);
  for (int m = 0; m < B; ++m) {
    const int r0 = b->h_ioff[m], r1 = r0 + b->h_ipad[m];
    rb_first[m] = (int)rb_mesh.size();
    for (int r = r0; r < r1; r += rows_per_block) {
      rb_mesh.push_back(m);
      rb_row0.push_back(r);
      rb_row1.push_back(std::min(r1, r + rows_per_block));
    }
    rb_count[m] = (int)rb_mesh.size() - rb_first[m];
    sl_first[m] = r0 / 32;
    sl_count[m] = (r1 - r0) / 32;
    for (int s = r0 / 32; s < r1 / 32; ++s) sl_mesh[s] = m;
    const int t0 = b->h_toff[m], t1 = b->h_toff[m + 1];
    tb_first[m] = (int)tb_mesh.size();
    for (int e = t0; e < t1; e += kTetBlock) {
      tb_mesh.push_back(m);
      tb_t0.push_back(e);
      tb_t1.push_back(std::min(t1, e + kTetBlock));
    }
    tb_count[m] = (int)tb_mesh.size() - tb_first[m];
  }
  BView& V = b->view;
  V.nmesh = B;
  V.nrb = (int)rb_mesh.size();
  V.ntb = (int)tb_mesh.size();
  mls_status st;
  int* p;
#define UP(field, vec) \
  if ((st = bupload(b, b->tables, &p, vec)) != MLS_OK) return st; \
  V.field = p;
  UP(rb_mesh, rb_mesh) UP(rb_row0, rb_row0) UP(rb_row1, rb_row1) UP(rb_first, rb_first) UP(rb_count, rb_count)
  UP(sl_mesh, sl_mesh) UP(sl_first, sl_first) UP(sl_count, sl_count)
  UP(tb_mesh, tb_mesh) UP(tb_t0, tb_t0) UP(tb_t1, tb_t1) UP(tb_first, tb_first) UP(tb_count, tb_count)
#undef UP
  // partials: row-block partials sized for this shape; energy partials for tets + row blocks
  if (b->part_rb) { cudaFree(b->part_rb); b->part_rb = nullptr; }
  if (b->part_e) { cudaFree(b->part_e); b->part_e = nullptr; }
  if (cudaMalloc(&b->part_rb, sizeof(double) * 4 * std::max(V.nrb, 1)) != cudaSuccess ||
      cudaMalloc(&b->part_e, sizeof(double) * 2 * std::max(V.nrb + V.ntb, 1)) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, MLS_ENOMEM, "batch partials");
  }
  V.part_rb = b->part_rb;
  V.part_tb = b->part_e;
  V.part_sl = b->part_sl;
  V.mass_min = b->mass_min;
  V.cnt = b->cnt;
  V.M = b->M;
  b->nrb = V.nrb;
  b->ntb = V.ntb;
  b->shape = sh;
  b->graph_dirty = true;
  return MLS_OK;
}

BParams params(mls_batch* b, double dt) {
  mls_ctx* c = b->ctx;
  BParams P{};
  // BDF2: Eq. IP with alpha = 4/9 is the implicit-Euler potential of the step 2 dt / 3
  P.h2 = b->bdf2 ? (2.0 * dt / 3.0) * (2.0 * dt / 3.0) : dt * dt;
  const double gm = std::sqrt(c->grav[0] * c->grav[0] + c->grav[1] * c->grav[1] + c->grav[2] * c->grav[2]);
  P.scale0 = dt * dt * std::max(gm, 1e-30);
  P.newton_tol = c->opt.newton_tol;
  P.pcg_rtol = c->opt.pcg_rtol;
  P.eta_floor = c->opt.precision == MLS_FP64 ? 1e-13 : 1e-6;
  P.max_newton = c->opt.max_newton;
  P.max_pcg = c->opt.max_pcg;
  P.kappa = c->kappa; P.dhat = c->dhat; P.po = c->po;
  P.pn0 = c->pn[0]; P.pn1 = c->pn[1]; P.pn2 = c->pn[2];
  P.contact = c->contact;
  P.fmu = c->contact ? c->fric_mu : 0.0;
  P.feps = c->fric_eps_v * dt;
  return P;
}

BEnergyIn energy_in(mls_ctx* c) {
  return BEnergyIn{c->t, c->tets, c->Dminv, c->vol, c->mu, c->lam, c->mass, c->pinned, c->xtil, c->xt};
}

template <typename VT, typename MT>
mls_status launch_cycle(mls_batch* b, cudaStream_t s, int first);

BBasisView bbasis(mls_ctx* c) {
  const Basis& B = c->basis;
  return BBasisView{B.vcoef, B.hcoef, B.vrow, B.vh, B.hrow, B.hv, B.rchunk_handle, B.rchunk_beg, B.rchunk_ptr,
                    B.rpart, B.rcount, B.nrchunk};
}

// one PCG iteration for every active mesh: product and direction update,
// vector update, and (two-level) the multiplicative cycle
template <typename VT, typename MT>
mls_status launch_pcg_iter(mls_batch* b, cudaStream_t s) {
  mls_ctx* c = b->ctx;
  const BView& V = b->view;
  const int ns = c->n_slices;
  const bool tl = b->two_level;
  const Vec4<VT>* zin = (const Vec4<VT>*)(tl ? c->vz2 : c->vz);
  cudaError_t e;
  if (b->shape.lanes == 8)
    e = launch_chained(k_bspmv<VT, MT, 8>, dim3(ns), dim3(256), s, V, c->n, (const int*)c->slice_ptr,
                       (const int*)c->col, (const int*)c->row_len, (const MT*)c->hval, zin, (Vec4<VT>*)c->vp,
                       (Vec4<VT>*)c->vq);
  else
    e = launch_chained(k_bspmv<VT, MT, 4>, dim3(ns), dim3(128), s, V, c->n, (const int*)c->slice_ptr,
                       (const int*)c->col, (const int*)c->row_len, (const MT*)c->hval, zin, (Vec4<VT>*)c->vp,
                       (Vec4<VT>*)c->vq);
  mls_status st = bcheck(b, e, "k_bspmv");
  if (st != MLS_OK) return st;
  st = bcheck(b, launch_chained(k_bupdate<VT>, dim3(V.nrb), dim3(b->shape.row_threads), s, V, c->opt.max_pcg,
                                tl ? 1 : 0, (VT)c->opt.omega, (const VT*)c->dinv, (Vec4<VT>*)c->vx,
                                (Vec4<VT>*)c->vr, (Vec4<VT>*)c->vz, (const Vec4<VT>*)c->vp,
                                (const Vec4<VT>*)c->vq), "k_bupdate");
  if (st != MLS_OK || !tl) return st;
  return launch_cycle<VT, MT>(b, s, 0);
}

// the symmetric multiplicative two-level cycle on r with the pre-smoothed
// z1 = omega D^{-1} r in vz: t = r - H z1; c = W^T W U^T t; z1 += U c;
// zf = z1 + omega D^{-1} (r - H z1) into vz2, with r.zf and beta
template <typename VT, typename MT>
mls_status launch_cycle(mls_batch* b, cudaStream_t s, int first) {
  mls_ctx* c = b->ctx;
  const BView& V = b->view;
  const int ns = c->n_slices;
  mls_status st = bcheck(b, launch_chained(k_bresidual<VT, MT>, dim3(ns), dim3(128), s, V, c->n,
                                           (const int*)c->slice_ptr, (const int*)c->col, (const int*)c->row_len,
                                           (const MT*)c->hval, (const Vec4<VT>*)c->vr, (const Vec4<VT>*)c->vz,
                                           (Vec4<VT>*)c->vw), "k_bresidual");
  if (st != MLS_OK) return st;
  const BBasisView BB = bbasis(c);
  if ((st = bcheck(b, launch_chained(k_brestrict<VT>, dim3((BB.nrchunk + 7) / 8), dim3(256), s, V, b->coarse, BB,
                                     (const Vec4<VT>*)c->vw, (VT*)c->cvec), "k_brestrict")) != MLS_OK)
    return st;
  const int rg = (b->coarse.r + 1) / 2;
  if ((st = bcheck(b, launch_chained(k_btrigemv<VT>, dim3(rg), dim3(256), s, V, b->coarse, (const VT*)b->WT, 2,
                                     (const VT*)c->cvec, (VT*)c->cvec2), "k_btrigemv")) != MLS_OK)
    return st;
  if ((st = bcheck(b, launch_chained(k_bprolong<VT>, dim3(V.nrb), dim3(b->shape.row_threads), s, V, BB,
                                     (const VT*)c->cvec2, (Vec4<VT>*)c->vz), "k_bprolong")) != MLS_OK)
    return st;
  return bcheck(b, launch_chained(k_bpost_smooth<VT, MT>, dim3(ns), dim3(128), s, V, first, (VT)c->opt.omega, c->n,
                                  (const int*)c->slice_ptr, (const int*)c->col, (const int*)c->row_len,
                                  (const MT*)c->hval, (const VT*)c->dinv, (const Vec4<VT>*)c->vr,
                                  (const Vec4<VT>*)c->vz, (Vec4<VT>*)c->vz2), "k_bpost_smooth");
}

// Galerkin operator of every mesh (dense product, block diagonal), its
// per-mesh float64 Cholesky and inverse factors
template <typename VT>
mls_status launch_coarse(mls_batch* b, cudaStream_t s) {
  mls_ctx* c = b->ctx;
  mls_status st = build_galerkin(c);
  if (st != MLS_OK) return bfail(b, st, mls_last_error(c));
  k_bchol<<<b->nmesh, 256, 0, s>>>(b->view, b->coarse, c->Ac, c->Acopy, b->coarse.r);
  k_btrinv<VT><<<b->nmesh, 256, 0, s>>>(b->view, b->coarse, c->Ac, c->Acopy, b->coarse.r, (VT*)b->W, (VT*)b->WT);
  return bcheck(b, cudaGetLastError(), "batched coarse factor");
}

template <typename VT>
mls_status launch_prep(mls_batch* b, cudaStream_t s, const BParams& P) {
  mls_ctx* c = b->ctx;
  k_bprep<VT><<<b->view.nrb, b->shape.row_threads, 0, s>>>(b->view, P, b->two_level ? 1 : 0, (VT)c->opt.omega,
                                                          c->grad, (const Vec4<VT>*)c->vb, (const VT*)c->dinv,
                                                          c->xk, c->xt, (Vec4<VT>*)c->vx, (Vec4<VT>*)c->vr,
                                                          (Vec4<VT>*)c->vz, (Vec4<VT>*)c->vp, (Vec4<VT>*)c->vq);
  return bcheck(b, cudaGetLastError(), "k_bprep");
}

template <typename VT>
mls_status launch_dir(mls_batch* b, cudaStream_t s, const BParams& P) {
  mls_ctx* c = b->ctx;
  k_bdir<VT><<<b->view.nrb, b->shape.row_threads, 0, s>>>(b->view, P, (const Vec4<VT>*)c->vx, c->pinned, c->grad,
                                                         c->xk, c->xt, c->dir);
  return bcheck(b, cudaGetLastError(), "k_bdir");
}

// Conditional handle for a WHILE node to be added to the graph that stream s
// is capturing into.  assign_default: the condition is reset to 1 at every
// launch of the graph (the outermost loop); otherwise a kernel captured
// before the node sets it.
mls_status make_handle(mls_batch* b, cudaStream_t s, bool assign_default, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  mls_status st = bcheck(b, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, nullptr, nullptr, nullptr), "capture info");
  if (st != MLS_OK) return st;
  return bcheck(b, cudaGraphConditionalHandleCreate(h, g, assign_default ? 1u : 0u,
                                                    assign_default ? cudaGraphCondAssignDefault : 0u),
                "conditional handle");
}

// Adds the WHILE node of handle h at the capture point of stream s and
// starts capturing its body into stream body.
mls_status begin_while(mls_batch* b, cudaStream_t s, cudaStream_t body, cudaGraphConditionalHandle h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  const cudaGraphEdgeData* edges = nullptr;
  size_t nd = 0;
  mls_status st = bcheck(b, cudaStreamGetCaptureInfo(s, &cs, nullptr, &g, &deps, &edges, &nd), "capture info");
  if (st != MLS_OK) return st;
  cudaGraphNodeParams cp{};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node;
  if ((st = bcheck(b, cudaGraphAddNode(&node, g, deps, edges, nd, &cp), "conditional node")) != MLS_OK) return st;
  if ((st = bcheck(b, cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies),
                   "capture dependencies")) != MLS_OK)
    return st;
  return bcheck(b, cudaStreamBeginCaptureToGraph(body, cp.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeRelaxed),
                "body capture");
}

mls_status end_body(mls_batch* b, cudaStream_t body) {
  cudaGraph_t g;
  return bcheck(b, cudaStreamEndCapture(body, &g), "body end");
}

void abandon_capture(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(s, &g);
    if (g) cudaGraphDestroy(g);
  }
  cudaGetLastError();
}

template <typename VT, typename MT>
mls_status capture_step(mls_batch* b, double dt) {
  mls_ctx* c = b->ctx;
  const BParams P = params(b, dt);
  const BEnergyIn EI = energy_in(c);
  cudaStream_t s0 = b->cap;
  cudaStream_t s1 = nullptr, s2 = nullptr;
  mls_status st = MLS_OK;
  if (cudaStreamCreateWithFlags(&s1, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    if (s1) cudaStreamDestroy(s1);
    return bfail(b, MLS_ECUDA, "capture streams");
  }
  cudaStream_t saved = c->stream;
  cudaGraph_t graph = nullptr;
  const BView& V = b->view;
  const int eb = V.ntb + V.nrb;
  const int rt = b->shape.row_threads;
  int* trips = b->trips;   // [0] PCG bodies, [1] line-search bodies, [2] Newton bodies, [3] loop entries
  // worst-case loop trips per timestep allowed by the per-mesh caps
  const int cap_newton = P.max_newton + 1;
  const int cap_pcg = std::min<int64_t>(INT32_MAX / 2, ((int64_t)P.max_pcg / 2 + 2) * cap_newton);
  const int cap_ls = 64 * cap_newton;
  const int cap_entry = 4 * cap_newton;
  auto run = [&]() -> mls_status {
    mls_status r;
    if ((r = bcheck(b, cudaStreamBeginCapture(s0, cudaStreamCaptureModeRelaxed), "begin capture")) != MLS_OK) return r;
    c->stream = s0;
    // predictor and start states
    k_breset<<<(b->nmesh + 127) / 128, 128, 0, s0>>>(b->nmesh, b->M);
    if ((r = b->bdf2 ? launch_predictor_bdf2(c, b->bx, b->bv, b->bxp, b->bvp, dt)
                     : launch_predictor(c, b->bx, b->bv, dt)) != MLS_OK)
      return r;
    k_benergy<0><<<eb, kTetBlock, 0, s0>>>(V, EI, P, c->xt, c->xt);
    k_benergy<1><<<eb, kTetBlock, 0, s0>>>(V, EI, P, c->xk, c->xk);
    k_bselect<<<V.nrb, rt, 0, s0>>>(V, c->xt, c->xk);
    if (b->two_level) {
      // coarse operators once per step, at the start iterate
      if ((r = launch_eval_elements(c, c->xk, nullptr)) != MLS_OK) return r;
      if ((r = launch_gather_grad(c, c->xk, c->dscal + 2)) != MLS_OK) return r;
      if ((r = launch_assemble(c, c->xk)) != MLS_OK) return r;
      if ((r = launch_coarse<VT>(b, s0)) != MLS_OK) return r;
    }
    // Newton loop: entered with its condition at 1 on every launch
    cudaGraphConditionalHandle hn, hp, hl;
    if ((r = make_handle(b, s0, true, &hn)) != MLS_OK) return r;
    if ((r = begin_while(b, s0, s1, hn)) != MLS_OK) return r;
    c->stream = s1;
    if ((r = launch_eval_elements(c, c->xk, nullptr)) != MLS_OK) return r;
    if ((r = launch_gather_grad(c, c->xk, c->dscal + 2)) != MLS_OK) return r;
    if ((r = launch_assemble(c, c->xk)) != MLS_OK) return r;
    if ((r = launch_prep<VT>(b, s1, P)) != MLS_OK) return r;
    if (b->two_level && (r = launch_cycle<VT, MT>(b, s1, 1)) != MLS_OK) return r;
    // PCG loop
    if ((r = make_handle(b, s1, false, &hp)) != MLS_OK) return r;
    k_bcond<<<1, 256, 0, s1>>>(b->nmesh, b->M, 0, P.max_newton, hp, 1, nullptr, trips + 3, cap_entry);
    if ((r = begin_while(b, s1, s2, hp)) != MLS_OK) return r;
    if ((r = launch_pcg_iter<VT, MT>(b, s2)) != MLS_OK) return r;
    if ((r = launch_pcg_iter<VT, MT>(b, s2)) != MLS_OK) return r;
    k_bcond<<<1, 256, 0, s2>>>(b->nmesh, b->M, 0, P.max_newton, hp, 1, nullptr, trips + 0, cap_pcg);
    if ((r = end_body(b, s2)) != MLS_OK) return r;
    if ((r = launch_dir<VT>(b, s1, P)) != MLS_OK) return r;
    // line-search loop
    if ((r = make_handle(b, s1, false, &hl)) != MLS_OK) return r;
    k_bcond<<<1, 256, 0, s1>>>(b->nmesh, b->M, 1, P.max_newton, hl, 1, nullptr, trips + 3, cap_entry);
    if ((r = begin_while(b, s1, s2, hl)) != MLS_OK) return r;
    k_benergy<2><<<eb, kTetBlock, 0, s2>>>(V, EI, P, c->xk, c->dir);
    k_bapply<<<V.nrb, rt, 0, s2>>>(V, c->xk, c->dir);
    k_bcond<<<1, 256, 0, s2>>>(b->nmesh, b->M, 1, P.max_newton, hl, 1, nullptr, trips + 1, cap_ls);
    if ((r = end_body(b, s2)) != MLS_OK) return r;
    k_bcond<<<1, 256, 0, s1>>>(b->nmesh, b->M, 2, P.max_newton, hn, 1, nullptr, trips + 2, cap_newton);
    if ((r = end_body(b, s1)) != MLS_OK) return r;
    c->stream = s0;
    return bcheck(b, cudaGetLastError(), "capture launches");
  };
  st = run();
  c->stream = saved;
  abandon_capture(s2);
  abandon_capture(s1);
  cudaError_t e = cudaStreamEndCapture(s0, &graph);
  if (st == MLS_OK && e != cudaSuccess) st = bcheck(b, e, "end capture");
  cudaGetLastError();
  if (st == MLS_OK) {
    if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
    st = bcheck(b, cudaGraphInstantiate(&b->exec, graph, 0), "graph instantiate");
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(s1);
  cudaStreamDestroy(s2);
  if (st == MLS_OK) {
    b->graph_dt = dt;
    b->graph_bdf2 = b->bdf2;
    b->graph_dirty = false;
    // kernels per body: Newton = element, gradient, assembly, PCG set-up,
    // two loop-entry conditions, direction, Newton condition (+ the first
    // cycle of five kernels with two levels); PCG = two iterations of two
    // kernels (+ five cycle kernels each) + condition; line search = energy,
    // apply, condition.  Outside the loops: reset, predictor, two energies,
    // select (+ element, gradient, assembly, three Galerkin kernels, the
    // per-mesh Cholesky and inverse with two levels).
    b->launches_fixed = b->two_level ? 5 + 3 + 3 + 2 : 5;
    b->launches_newton = b->two_level ? 8 + 5 : 8;
    b->launches_pcg = b->two_level ? 2 * 7 + 1 : 5;
    b->launches_ls = 3;
  }
  return st;
}

// Times the PCG iteration of every candidate shape on the assembled system
// of the current state and keeps the fastest.
template <typename VT, typename MT>
mls_status autotune(mls_batch* b, double dt) {
  mls_ctx* c = b->ctx;
  const BParams P = params(b, dt);
  const BEnergyIn EI = energy_in(c);
  cudaStream_t s = b->cap;
  cudaStream_t saved = c->stream;
  c->stream = s;
  mls_status st;
  // one assembled system from the predictor (meshes with an infeasible
  // predictor are timed on it all the same)
  if ((st = launch_predictor(c, b->bx, b->bv, dt)) != MLS_OK) { c->stream = saved; return st; }
  if ((st = launch_eval_elements(c, c->xk, nullptr)) != MLS_OK) { c->stream = saved; return st; }
  if ((st = launch_gather_grad(c, c->xk, c->dscal + 2)) != MLS_OK) { c->stream = saved; return st; }
  if ((st = launch_assemble(c, c->xk)) != MLS_OK) { c->stream = saved; return st; }
  (void)EI;
  if (b->two_level) {
    k_breset<<<(b->nmesh + 127) / 128, 128, 0, s>>>(b->nmesh, b->M);
    if ((st = launch_coarse<VT>(b, s)) != MLS_OK) { c->stream = saved; return st; }
    b->galerkin_warm = true;
  }
  const BShape cands[] = {{4, 256, 1}, {4, 128, 1}, {4, 256, 2}, {4, 512, 1}, {8, 256, 1}, {8, 128, 1}, {8, 256, 2}};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  BShape win = cands[0];
  BParams Pt = P;
  Pt.pcg_rtol = 0.0;        // no mesh converges while timing
  Pt.eta_floor = 0.0;
  Pt.newton_tol = 0.0;
  for (const BShape& sh : cands) {
    if ((st = build_tables(b, sh)) != MLS_OK) break;
    k_breset<<<(b->nmesh + 127) / 128, 128, 0, s>>>(b->nmesh, b->M);
    if ((st = launch_prep<VT>(b, s, Pt)) != MLS_OK) break;
    for (int w = 0; w < 2; ++w)
      if ((st = launch_pcg_iter<VT, MT>(b, s)) != MLS_OK) break;
    if (st != MLS_OK) break;
    cudaEventRecord(e0, s);
    for (int it = 0; it < 8; ++it)
      if ((st = launch_pcg_iter<VT, MT>(b, s)) != MLS_OK) break;
    if (st != MLS_OK) break;
    cudaEventRecord(e1, s);
    if ((st = bcheck(b, cudaEventSynchronize(e1), "autotune sync")) != MLS_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    b->tune_ms += ms;
    if (ms < best) { best = ms; win = sh; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->stream = saved;
  if (st != MLS_OK) return st;
  if ((st = build_tables(b, win)) != MLS_OK) return st;
  b->tuned = true;
  return MLS_OK;
}

template <typename VT, typename MT>
mls_status batch_step_t(mls_batch* b, const double* x, const double* v, const double* xp, const double* vp,
                        double dt, double* dx) {
  mls_ctx* c = b->ctx;
  mls_status st;
  cudaStream_t user = c->stream;
  // order the internal stream after the caller's stream
  cudaEvent_t ev;
  if ((st = bcheck(b, cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event")) != MLS_OK) return st;
  cudaEventRecord(ev, user);
  cudaStreamWaitEvent(b->cap, ev, 0);
  k_bpack<<<(b->n + 255) / 256, 256, 0, b->cap>>>(b->n, b->vmap, x, v, b->bx, b->bv,
                                                  c->pn[0] * (c->po + 1e3), c->pn[1] * (c->po + 1e3),
                                                  c->pn[2] * (c->po + 1e3));
  if ((st = bcheck(b, cudaGetLastError(), "k_bpack")) != MLS_OK) { cudaEventDestroy(ev); return st; }
  if (b->bdf2) {
    k_bpack<<<(b->n + 255) / 256, 256, 0, b->cap>>>(b->n, b->vmap, xp, vp, b->bxp, b->bvp,
                                                    c->pn[0] * (c->po + 1e3), c->pn[1] * (c->po + 1e3),
                                                    c->pn[2] * (c->po + 1e3));
    if ((st = bcheck(b, cudaGetLastError(), "k_bpack history")) != MLS_OK) { cudaEventDestroy(ev); return st; }
  }
  if (b->two_level && !b->has_basis) {
    cudaEventDestroy(ev);
    return bfail(b, MLS_EINVAL, "two-level batch: upload the per-mesh bases first");
  }
  if (!b->tuned) {
    if ((st = autotune<VT, MT>(b, dt)) != MLS_OK) { cudaEventDestroy(ev); return st; }
  }
  if (b->two_level && !b->galerkin_warm) {
    // first Galerkin product outside capture (it allocates its row table)
    cudaStream_t saved = c->stream;
    c->stream = b->cap;
    st = build_galerkin(c);
    c->stream = saved;
    if (st != MLS_OK) { cudaEventDestroy(ev); return bfail(b, st, mls_last_error(c)); }
    b->galerkin_warm = true;
  }
  if (b->graph_dirty || b->graph_dt != dt || b->graph_bdf2 != b->bdf2 || !b->exec) {
    if ((st = capture_step<VT, MT>(b, dt)) != MLS_OK) { cudaEventDestroy(ev); return st; }
  }
  cudaMemsetAsync(b->trips, 0, sizeof(int) * 4, b->cap);
  if ((st = bcheck(b, cudaGraphLaunch(b->exec, b->cap), "graph launch")) != MLS_OK) { cudaEventDestroy(ev); return st; }
  k_bunpack<<<(b->n + 255) / 256, 256, 0, b->cap>>>(b->n, b->vmap, c->xk, c->xt, dx);
  cudaMemcpyAsync(b->h_M, b->M, sizeof(BMesh) * b->nmesh, cudaMemcpyDeviceToHost, b->cap);
  cudaMemcpyAsync(b->h_trips, b->trips, sizeof(int) * 4, cudaMemcpyDeviceToHost, b->cap);
  cudaEventRecord(ev, b->cap);
  cudaStreamWaitEvent(user, ev, 0);
  st = bcheck(b, cudaStreamSynchronize(b->cap), "batch step");
  cudaEventDestroy(ev);
  return st;
}

}  // namespace

extern "C" {

mls_status mls_batch_create(mls_batch** out, const mls_options* opt) {
  if (!out) return MLS_EINVAL;
  *out = nullptr;
  mls_options o;
  if (opt) o = *opt;
  else mls_default_options(&o);
  if (o.preconditioner != MLS_PRECOND_BLOCK_JACOBI && o.preconditioner != MLS_PRECOND_TWO_LEVEL) return MLS_EINVAL;
  if (!(o.omega > 0.0)) return MLS_EINVAL;  // the automatic damping is a single-mesh option
  mls_batch* b = new (std::nothrow) mls_batch();
  if (!b) return MLS_ENOMEM;
  mls_status st = mls_create(&b->ctx, &o);
  if (st != MLS_OK) { delete b; return st; }
  b->two_level = o.preconditioner == MLS_PRECOND_TWO_LEVEL;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    mls_destroy(b->ctx);
    delete b;
    return MLS_ECUDA;
  }
  *out = b;
  return MLS_OK;
}

mls_status mls_batch_destroy(mls_batch* b) {
  if (!b) return MLS_OK;
  if (b->cap) cudaStreamSynchronize(b->cap);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  free_tables(b);
  for (void* p : b->coarse_alloc) cudaFree(p);
  if (b->W) cudaFree(b->W);
  if (b->WT) cudaFree(b->WT);
  for (void* p : {(void*)b->vmap, (void*)b->bx, (void*)b->bv, (void*)b->bxp, (void*)b->bvp, (void*)b->M,
                  (void*)b->trips, (void*)b->any,
                  (void*)b->mass_min, (void*)b->cnt, (void*)b->part_rb, (void*)b->part_sl, (void*)b->part_e})
    if (p) cudaFree(p);
  if (b->h_M) cudaFreeHost(b->h_M);
  if (b->h_trips) cudaFreeHost(b->h_trips);
  if (b->cap) cudaStreamDestroy(b->cap);
  mls_destroy(b->ctx);
  delete b;
  return MLS_OK;
}

const char* mls_batch_last_error(const mls_batch* b) {
  if (!b) return "null batch";
  return b->err.empty() ? mls_last_error(b->ctx) : b->err.c_str();
}

mls_status mls_batch_upload(mls_batch* b, int32_t n_meshes, const int32_t* vert_offsets, const int32_t* tet_offsets,
                            const double* rest_xyz, const int32_t* tets, const double* youngs,
                            const double* poisson, const double* density, const uint8_t* dirichlet) {
  if (!b) return MLS_EINVAL;
  b->err.clear();
  if (n_meshes < 1 || !vert_offsets || !tet_offsets || !rest_xyz || !tets || !youngs || !poisson || !density)
    return bfail(b, MLS_EINVAL, "batch upload: no meshes or a null array");
  if (vert_offsets[0] != 0 || tet_offsets[0] != 0) return bfail(b, MLS_EINVAL, "batch upload: offsets must start at 0");
  for (int m = 0; m < n_meshes; ++m)
    if (vert_offsets[m + 1] <= vert_offsets[m] || tet_offsets[m + 1] <= tet_offsets[m])
      return bfail(b, MLS_EINVAL, "batch upload: mesh " + std::to_string(m) + " is empty");
  const int nu = vert_offsets[n_meshes], nt = tet_offsets[n_meshes];
  // tets reference vertices of their own mesh only
  for (int m = 0; m < n_meshes; ++m)
    for (int64_t k = 4 * (int64_t)tet_offsets[m]; k < 4 * (int64_t)tet_offsets[m + 1]; ++k)
      if (tets[k] < vert_offsets[m] || tets[k] >= vert_offsets[m + 1])
        return bfail(b, MLS_EINVAL, "batch upload: a tet of mesh " + std::to_string(m) + " references another mesh");
  // padded internal layout
  std::vector<int> ioff(n_meshes), ipad(n_meshes);
  int n = 0;
  for (int m = 0; m < n_meshes; ++m) {
    const int nv = vert_offsets[m + 1] - vert_offsets[m];
    ioff[m] = n;
    ipad[m] = (nv + 31) / 32 * 32;
    n += ipad[m];
  }
  std::vector<double> X(3 * (size_t)n, 0.0);
  std::vector<uint8_t> pin(n, 1);
  std::vector<int> vmap(n, -1);
  for (int m = 0; m < n_meshes; ++m)
    for (int u = vert_offsets[m]; u < vert_offsets[m + 1]; ++u) {
      const int i = ioff[m] + (u - vert_offsets[m]);
      vmap[i] = u;
      for (int k = 0; k < 3; ++k) X[3 * (size_t)i + k] = rest_xyz[3 * (size_t)u + k];
      pin[i] = dirichlet ? (dirichlet[u] ? 1 : 0) : 0;
    }
  for (int m = 0; m < n_meshes; ++m)   // dummy rows: rest at the mesh's first vertex
    for (int i = ioff[m] + vert_offsets[m + 1] - vert_offsets[m]; i < ioff[m] + ipad[m]; ++i)
      for (int k = 0; k < 3; ++k) X[3 * (size_t)i + k] = rest_xyz[3 * (size_t)vert_offsets[m] + k];
  std::vector<int> T(4 * (size_t)nt);
  for (int m = 0; m < n_meshes; ++m)
    for (int64_t k = 4 * (int64_t)tet_offsets[m]; k < 4 * (int64_t)tet_offsets[m + 1]; ++k)
      T[k] = ioff[m] + (tets[k] - vert_offsets[m]);
  mls_status st = mls_upload_mesh(b->ctx, n, X.data(), nt, T.data(), youngs, poisson, density, pin.data());
  if (st != MLS_OK) return bfail(b, st, std::string("batch upload: ") + mls_last_error(b->ctx));
  // per-mesh smallest free-vertex lumped mass
  std::vector<double> mass(n, 0.0);
  for (int e = 0; e < nt; ++e) {
    const double* p0 = X.data() + 3 * (size_t)T[4 * e];
    double D[3][3];
    for (int k = 0; k < 3; ++k)
      for (int a = 0; a < 3; ++a) D[a][k] = X[3 * (size_t)T[4 * e + k + 1] + a] - p0[a];
    const double det = D[0][0] * (D[1][1] * D[2][2] - D[1][2] * D[2][1]) - D[0][1] * (D[1][0] * D[2][2] - D[1][2] * D[2][0]) +
                       D[0][2] * (D[1][0] * D[2][1] - D[1][1] * D[2][0]);
    for (int a = 0; a < 4; ++a) mass[T[4 * e + a]] += density[e] * det / 24.0;
  }
  std::vector<double> mmin(n_meshes, 0.0);
  for (int m = 0; m < n_meshes; ++m) {
    double lo = 1e300;
    for (int i = ioff[m]; i < ioff[m] + vert_offsets[m + 1] - vert_offsets[m]; ++i)
      if (!pin[i]) lo = std::min(lo, mass[i]);
    mmin[m] = lo < 1e300 ? lo : 0.0;
  }
  // (re)allocate batch state
  for (void** p : {(void**)&b->vmap, (void**)&b->bx, (void**)&b->bv, (void**)&b->bxp, (void**)&b->bvp,
                   (void**)&b->M, (void**)&b->trips,
                   (void**)&b->any, (void**)&b->mass_min, (void**)&b->cnt, (void**)&b->part_sl})
    if (*p) { cudaFree(*p); *p = nullptr; }
  if (b->h_M) { cudaFreeHost(b->h_M); b->h_M = nullptr; }
  if (b->h_trips) { cudaFreeHost(b->h_trips); b->h_trips = nullptr; }
  bool ok = cudaMalloc(&b->vmap, sizeof(int) * n) == cudaSuccess &&
            cudaMalloc(&b->bx, sizeof(double) * 3 * n) == cudaSuccess &&
            cudaMalloc(&b->bv, sizeof(double) * 3 * n) == cudaSuccess &&
            cudaMalloc(&b->M, sizeof(BMesh) * n_meshes) == cudaSuccess &&
            cudaMalloc(&b->trips, sizeof(int) * 4) == cudaSuccess &&
            cudaMalloc(&b->any, sizeof(int)) == cudaSuccess &&
            cudaMalloc(&b->mass_min, sizeof(double) * n_meshes) == cudaSuccess &&
            cudaMalloc(&b->cnt, sizeof(unsigned) * BC_COUNT * n_meshes) == cudaSuccess &&
            cudaMalloc(&b->part_sl, sizeof(double) * (n / 32)) == cudaSuccess &&
            cudaMallocHost(&b->h_M, sizeof(BMesh) * n_meshes) == cudaSuccess &&
            cudaMallocHost(&b->h_trips, sizeof(int) * 4) == cudaSuccess;
  if (!ok) { cudaGetLastError(); return bfail(b, MLS_ENOMEM, "batch state allocation"); }
  if ((st = bcheck(b, cudaMemcpy(b->vmap, vmap.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "vmap")) != MLS_OK) return st;
  if ((st = bcheck(b, cudaMemcpy(b->mass_min, mmin.data(), sizeof(double) * n_meshes, cudaMemcpyHostToDevice), "mass")) != MLS_OK) return st;
  if ((st = bcheck(b, cudaMemset(b->cnt, 0, sizeof(unsigned) * BC_COUNT * n_meshes), "counters")) != MLS_OK) return st;
  b->nmesh = n_meshes;
  b->n_user = nu;
  b->n = n;
  b->h_voff.assign(vert_offsets, vert_offsets + n_meshes + 1);
  b->h_toff.assign(tet_offsets, tet_offsets + n_meshes + 1);
  b->h_ioff = ioff;
  b->h_ipad = ipad;
  b->h_vmap = vmap;
  b->has_basis = false;
  b->galerkin_warm = false;
  b->tuned = false;
  b->tune_ms = 0.0;
  if ((st = build_tables(b, BShape{})) != MLS_OK) return st;
  return MLS_OK;
}

mls_status mls_batch_upload_basis(mls_batch* b, int32_t n_handles, const int32_t* handle_offsets,
                                  const double* origins, const int32_t* vrow, const int32_t* handle,
                                  const double* phi) {
  if (!b) return MLS_EINVAL;
  b->err.clear();
  if (b->nmesh < 1) return bfail(b, MLS_EINVAL, "batch basis: upload the meshes first");
  if (n_handles < 1 || !handle_offsets || !origins || !vrow || !handle || !phi)
    return bfail(b, MLS_EINVAL, "batch basis: no handles or a null array");
  const int B = b->nmesh;
  if (handle_offsets[0] != 0 || handle_offsets[B] != n_handles)
    return bfail(b, MLS_EINVAL, "batch basis: handle offsets must run from 0 to n_handles");
  for (int m = 0; m < B; ++m) {
    const int hm = handle_offsets[m + 1] - handle_offsets[m];
    if (hm < 1 || 12 * hm > kMaxCoarseRows)
      return bfail(b, MLS_EINVAL, "batch basis: mesh " + std::to_string(m) + " needs 1 to " +
                                      std::to_string(kMaxCoarseRows / 12) + " handles");
  }
  const int nu = b->n_user;
  if (vrow[0] != 0) return bfail(b, MLS_EINVAL, "batch basis: vrow must start at 0");
  for (int u = 0; u < nu; ++u)
    if (vrow[u + 1] < vrow[u]) return bfail(b, MLS_EINVAL, "batch basis: vrow must be non-decreasing");
  // every vertex's handles belong to its own mesh
  for (int m = 0; m < B; ++m)
    for (int u = b->h_voff[m]; u < b->h_voff[m + 1]; ++u)
      for (int k = vrow[u]; k < vrow[u + 1]; ++k)
        if (handle[k] < handle_offsets[m] || handle[k] >= handle_offsets[m + 1])
          return bfail(b, MLS_EINVAL, "batch basis: a vertex of mesh " + std::to_string(m) +
                                          " references a handle of another mesh");
  // internal (padded) vertex numbering
  std::vector<int> ivrow(b->n + 1, 0), ih;
  std::vector<double> iphi;
  ih.reserve(vrow[nu]);
  iphi.reserve(vrow[nu]);
  for (int i = 0; i < b->n; ++i) {
    const int u = b->h_vmap[i];
    if (u >= 0)
      for (int k = vrow[u]; k < vrow[u + 1]; ++k) { ih.push_back(handle[k]); iphi.push_back(phi[k]); }
    ivrow[i + 1] = (int)ih.size();
  }
  mls_status st = mls_upload_basis(b->ctx, n_handles, origins, ivrow.data(), ih.data(), iphi.data());
  if (st != MLS_OK) return bfail(b, st, std::string("batch basis: ") + mls_last_error(b->ctx));
  // block-diagonal coarse layout
  for (void* p : b->coarse_alloc) cudaFree(p);
  b->coarse_alloc.clear();
  if (b->W) { cudaFree(b->W); b->W = nullptr; }
  if (b->WT) { cudaFree(b->WT); b->WT = nullptr; }
  std::vector<int> coff(B), csz(B), crow(12 * n_handles), hmesh(n_handles);
  std::vector<int64_t> woff(B);
  int64_t wtot = 0;
  for (int m = 0; m < B; ++m) {
    coff[m] = 12 * handle_offsets[m];
    csz[m] = 12 * (handle_offsets[m + 1] - handle_offsets[m]);
    woff[m] = wtot;
    wtot += (int64_t)csz[m] * csz[m];
    for (int j = handle_offsets[m]; j < handle_offsets[m + 1]; ++j) hmesh[j] = m;
    for (int g = coff[m]; g < coff[m] + csz[m]; ++g) crow[g] = m;
  }
  BCoarse& C = b->coarse;
  C.r = 12 * n_handles;
  int* p;
  int64_t* q;
  if ((st = bupload(b, b->coarse_alloc, &p, coff)) != MLS_OK) return st;
  C.coff = p;
  if ((st = bupload(b, b->coarse_alloc, &p, csz)) != MLS_OK) return st;
  C.csz = p;
  if ((st = bupload(b, b->coarse_alloc, &q, woff)) != MLS_OK) return st;
  C.woff = q;
  if ((st = bupload(b, b->coarse_alloc, &p, crow)) != MLS_OK) return st;
  C.crow_mesh = p;
  if ((st = bupload(b, b->coarse_alloc, &p, hmesh)) != MLS_OK) return st;
  C.hmesh = p;
  const size_t vb = b->ctx->opt.precision == MLS_FP64 ? sizeof(double) : sizeof(float);
  if (cudaMalloc(&b->W, vb * wtot) != cudaSuccess || cudaMalloc(&b->WT, vb * wtot) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, MLS_ENOMEM, "batch basis: inverse factors");
  }
  b->has_basis = true;
  b->galerkin_warm = false;
  b->tuned = false;
  b->graph_dirty = true;
  return MLS_OK;
}

mls_status mls_batch_set_forces(mls_batch* b, const double* gravity, int contact, const double* plane_n,
                                double plane_o, double dhat, double kappa) {
  if (!b) return MLS_EINVAL;
  mls_status st = mls_set_forces(b->ctx, gravity, contact, plane_n, plane_o, dhat, kappa);
  if (st != MLS_OK) return bfail(b, st, mls_last_error(b->ctx));
  b->graph_dirty = true;
  return MLS_OK;
}

mls_status mls_batch_set_friction(mls_batch* b, double mu, double eps_v) {
  if (!b) return MLS_EINVAL;
  mls_status st = mls_set_friction(b->ctx, mu, eps_v);
  if (st != MLS_OK) return bfail(b, st, mls_last_error(b->ctx));
  b->graph_dirty = true;
  return MLS_OK;
}

mls_status mls_batch_retune(mls_batch* b) {
  if (!b) return MLS_EINVAL;
  b->tuned = false;
  b->tune_ms = 0.0;
  b->graph_dirty = true;
  return MLS_OK;
}

// one step of every mesh: implicit Euler (xp = vp = NULL) or BDF2 from the
// history (xp, vp) = (x^{t-1}, v^{t-1})
static mls_status batch_step_entry(mls_batch* b, const double* x, const double* v, const double* xp,
                                   const double* vp, double dt, double* dx_out, mls_batch_mesh_stats* stats,
                                   mls_batch_info* info) {
  if (!b) return MLS_EINVAL;
  b->err.clear();
  if (b->nmesh < 1) return bfail(b, MLS_EINVAL, "no meshes uploaded");
  if (!x || !v || !dx_out) return bfail(b, MLS_EINVAL, "null state pointer");
  if (!(dt > 0)) return bfail(b, MLS_EINVAL, "dt must be positive");
  const bool bdf2 = xp != nullptr;
  if (bdf2 && !b->bxp) {
    if (cudaMalloc(&b->bxp, sizeof(double) * 3 * b->n) != cudaSuccess ||
        cudaMalloc(&b->bvp, sizeof(double) * 3 * b->n) != cudaSuccess) {
      cudaGetLastError();
      if (b->bxp) { cudaFree(b->bxp); b->bxp = nullptr; }
      return bfail(b, MLS_ENOMEM, "BDF2 history buffers");
    }
  }
  b->bdf2 = bdf2;
  b->ctx->h = bdf2 ? 2.0 * dt / 3.0 : dt;
  b->ctx->h_step = dt;
  mls_status st;
  switch (b->ctx->opt.precision) {
    case MLS_FP64: st = batch_step_t<double, double>(b, x, v, xp, vp, dt, dx_out); break;
    case MLS_MIXED_FP32: st = batch_step_t<float, float>(b, x, v, xp, vp, dt, dx_out); break;
    default: st = batch_step_t<float, __nv_bfloat16>(b, x, v, xp, vp, dt, dx_out); break;
  }
  if (st != MLS_OK) return st;
  mls_status worst = MLS_OK;
  for (int m = 0; m < b->nmesh; ++m) {
    const BMesh& s = b->h_M[m];
    if (stats) {
      stats[m].status = s.status;
      stats[m].newton_iters = s.newton;
      stats[m].pcg_iters = s.pcg;
      stats[m].line_search_trials = s.trials;
      stats[m].step_rel = s.step_rel;
      stats[m].grad_norm = s.gnorm;
      stats[m].energy = s.E0;
    }
    if (s.status != MLS_OK && worst == MLS_OK) worst = (mls_status)s.status;
  }
  if (info) {
    const int* t = b->h_trips;
    // graph nodes run: fixed part + per Newton body (element, gradient,
    // assembly, prep, PCG condition, direction, Newton condition) + per PCG
    // body + per line-search body
    info->kernel_launches = 2 + b->launches_fixed + (int64_t)t[2] * b->launches_newton +
                            (int64_t)t[0] * b->launches_pcg + (int64_t)t[1] * b->launches_ls;
    info->graph_launches = 1;
    info->newton_rounds = t[2];
    info->pcg_rounds = t[0];
    info->line_search_rounds = t[1];
    info->spmv_lanes = b->shape.lanes;
    info->row_threads = b->shape.row_threads;
    info->rows_per_thread = b->shape.rows_per_thread;
    info->tune_ms = b->tune_ms;
  }
  if (worst != MLS_OK) {
    if (worst == MLS_ENOTCONV) b->err = "a mesh reached its Newton iteration cap";
    else b->err = "a mesh failed (see the per-mesh status)";
  }
  return worst;
}

mls_status mls_batch_step(mls_batch* b, const double* x, const double* v, double dt, double* dx_out,
                          mls_batch_mesh_stats* stats, mls_batch_info* info) {
  return batch_step_entry(b, x, v, nullptr, nullptr, dt, dx_out, stats, info);
}

mls_status mls_batch_step_bdf2(mls_batch* b, const double* x, const double* v, const double* x_prev,
                               const double* v_prev, double dt, double* dx_out, mls_batch_mesh_stats* stats,
                               mls_batch_info* info) {
  if (!b) return MLS_EINVAL;
  if (!x_prev || !v_prev) return bfail(b, MLS_EINVAL, "null history pointer");
  return batch_step_entry(b, x, v, x_prev, v_prev, dt, dx_out, stats, info);
}

}  // extern "C"
