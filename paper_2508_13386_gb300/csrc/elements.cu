// Per-tet Neo-Hookean energy, gradient and PSD-projected Hessian (the
// material model of Sec. 4: non-inverting Neo-Hookean, psi = mu/2 (|F|^2 - 3)
// - mu ln J + lam/2 ln^2 J), the point-plane barrier terms of Eq. IP, the
// line-search energy (with the lagged friction term D when it is on) and the
// point-plane CCD bound (Sec. 3.9).
//
// Hessian projection.  dP/dF of an isotropic energy is block diagonal in the
// frame of the SVD F = U diag(s) V^T.  Writing c3 = lam ln J - mu:
//   * for each pair i < k, the "twist" and "flip" directions
//     (u_i v_k^T -/+ u_k v_i^T)/sqrt2 have eigenvalues mu + c3/(s_i s_k) and
//     mu - c3/(s_i s_k);
//   * the three "scaling" directions u_i v_i^T span the 3x3 block
//     A3 = mu I + lam w w^T - c3 diag(w_i^2), w_i = 1/s_i.
// The projected dP/dF clamps negative eigenvalues to zero.  Mapping through
// B = dvec(F)/dx turns u_i v_k^T into the 12-vector u_i (x) nu_k with
// nu_k[a] = v_k . Dm^{-1}[a-1, :] (a = 1..3) and nu_k[0] = -sum_a nu_k[a], so
// each 3x3 block (a, b) of vol B^T [dP/dF]_+ B is U K_ab U^T with a 3x3 K_ab
// built from the clamped eigenvalues and nu.  This replaces a 9x9 or 12x12
// eigensolve by two 3x3 symmetric Jacobi eigensolves per tet.
#include "mls_internal.cuh"

namespace mls {

// ---- small dense helpers ------------------------------------------------------

// Cyclic Jacobi eigen-decomposition of a symmetric 3x3 A (overwritten by its
// diagonalised form); Q accumulates the rotations, so A_in = Q diag(A) Q^T.
template <typename T>
__device__ __forceinline__ void sym_eig3(T (&A)[3][3], T (&Q)[3][3], int sweeps) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) Q[i][j] = (i == j) ? T(1) : T(0);
  for (int s = 0; s < sweeps; ++s) {
#pragma unroll
    for (int pair = 0; pair < 3; ++pair) {
      const int p = pair == 2 ? 1 : 0;
      const int q = pair == 0 ? 1 : 2;
      const T apq = A[p][q];
      const T scale = fabs(A[p][p]) + fabs(A[q][q]);
      if (!(fabs(apq) > (sizeof(T) == 8 ? T(1e-300) : T(1e-30)) + scale * (sizeof(T) == 8 ? T(1e-17) : T(1e-9)))) continue;
      const T tau = (A[q][q] - A[p][p]) / (T(2) * apq);
      const T tt = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
      const T c = T(1) / sqrt(T(1) + tt * tt);
      const T sn = tt * c;
      // A <- J^T A J, J = [[c, s], [-s, c]] in the (p, q) plane
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T akp = A[k][p], akq = A[k][q];
        A[k][p] = c * akp - sn * akq;
        A[k][q] = sn * akp + c * akq;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T apk = A[p][k], aqk = A[q][k];
        A[p][k] = c * apk - sn * aqk;
        A[q][k] = sn * apk + c * aqk;
      }
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const T qkp = Q[k][p], qkq = Q[k][q];
        Q[k][p] = c * qkp - sn * qkq;
        Q[k][q] = sn * qkp + c * qkq;
      }
    }
  }
}

// SVD of F with det(U) = det(V) = +1 (valid for det F > 0): U and V as
// columns u_i, v_i; singular values s.
template <typename T>
__device__ __forceinline__ void svd3(const T (&F)[3][3], T (&U)[3][3], T (&s)[3], T (&V)[3][3]) {
  T A[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) A[i][j] = F[0][i] * F[0][j] + F[1][i] * F[1][j] + F[2][i] * F[2][j];
  sym_eig3<T>(A, V, sizeof(T) == 8 ? 6 : 5);
  // order eigenvalues descending (swap columns of V together with A's diagonal)
  T e0 = A[0][0], e1 = A[1][1], e2 = A[2][2];
#define MLS_SWAPCOL(a, b, ea, eb)                       \
  if (ea < eb) {                                        \
    T tmp = ea; ea = eb; eb = tmp;                      \
    _Pragma("unroll") for (int r = 0; r < 3; ++r) {     \
      T tv = V[r][a]; V[r][a] = V[r][b]; V[r][b] = tv;  \
    }                                                   \
  }
  MLS_SWAPCOL(0, 1, e0, e1)
  MLS_SWAPCOL(0, 2, e0, e2)
  MLS_SWAPCOL(1, 2, e1, e2)
#undef MLS_SWAPCOL
  const T detV = V[0][0] * (V[1][1] * V[2][2] - V[1][2] * V[2][1]) -
                 V[0][1] * (V[1][0] * V[2][2] - V[1][2] * V[2][0]) +
                 V[0][2] * (V[1][0] * V[2][1] - V[1][1] * V[2][0]);
  if (detV < T(0)) {
#pragma unroll
    for (int r = 0; r < 3; ++r) V[r][2] = -V[r][2];
  }
  T b[3][3];  // b_i = F v_i
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int r = 0; r < 3; ++r) b[i][r] = F[r][0] * V[0][i] + F[r][1] * V[1][i] + F[r][2] * V[2][i];
  T n0 = sqrt(b[0][0] * b[0][0] + b[0][1] * b[0][1] + b[0][2] * b[0][2]);
  T u0[3] = {b[0][0] / n0, b[0][1] / n0, b[0][2] / n0};
  T d01 = u0[0] * b[1][0] + u0[1] * b[1][1] + u0[2] * b[1][2];
  T w1[3] = {b[1][0] - d01 * u0[0], b[1][1] - d01 * u0[1], b[1][2] - d01 * u0[2]};
  T n1 = sqrt(w1[0] * w1[0] + w1[1] * w1[1] + w1[2] * w1[2]);
  T u1[3];
  if (n1 > n0 * (sizeof(T) == 8 ? T(1e-14) : T(1e-6))) {
    u1[0] = w1[0] / n1; u1[1] = w1[1] / n1; u1[2] = w1[2] / n1;
  } else {  // any unit vector orthogonal to u0
    T a[3] = {T(0), T(0), T(0)};
    a[fabs(u0[0]) < T(0.6) ? 0 : (fabs(u0[1]) < T(0.6) ? 1 : 2)] = T(1);
    T da = a[0] * u0[0] + a[1] * u0[1] + a[2] * u0[2];
    T c[3] = {a[0] - da * u0[0], a[1] - da * u0[1], a[2] - da * u0[2]};
    T nc = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
    u1[0] = c[0] / nc; u1[1] = c[1] / nc; u1[2] = c[2] / nc;
  }
  T u2[3] = {u0[1] * u1[2] - u0[2] * u1[1], u0[2] * u1[0] - u0[0] * u1[2], u0[0] * u1[1] - u0[1] * u1[0]};
  s[0] = n0;
  s[1] = u1[0] * b[1][0] + u1[1] * b[1][1] + u1[2] * b[1][2];
  s[2] = u2[0] * b[2][0] + u2[1] * b[2][1] + u2[2] * b[2][2];
#pragma unroll
  for (int r = 0; r < 3; ++r) { U[r][0] = u0[r]; U[r][1] = u1[r]; U[r][2] = u2[r]; }
}

// ---- element kernel -------------------------------------------------------------

struct ElemIn {
  int t;
  const int* __restrict__ tets;
  const double* __restrict__ Dminv;
  const double* __restrict__ vol;
  const double* __restrict__ mu;
  const double* __restrict__ lam;
};

__device__ __forceinline__ void load_tet(const ElemIn& in, int e, const Vec4d* __restrict__ x,
                                         double (&F)[3][3], double (&Dm)[3][3], int (&vid)[4]) {
  const int t = in.t;
#pragma unroll
  for (int a = 0; a < 4; ++a) vid[a] = in.tets[a * t + e];
  Vec4d p[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) p[a] = x[vid[a]];
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int b = 0; b < 3; ++b) Dm[k][b] = in.Dminv[(3 * k + b) * t + e];
  double Ds[3][3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    Ds[0][k] = p[k + 1].x - p[0].x;
    Ds[1][k] = p[k + 1].y - p[0].y;
    Ds[2][k] = p[k + 1].z - p[0].z;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) F[a][b] = Ds[a][0] * Dm[0][b] + Ds[a][1] * Dm[1][b] + Ds[a][2] * Dm[2][b];
}

__device__ __forceinline__ double det3(const double (&F)[3][3]) {
  return F[0][0] * (F[1][1] * F[2][2] - F[1][2] * F[2][1]) -
         F[0][1] * (F[1][0] * F[2][2] - F[1][2] * F[2][0]) +
         F[0][2] * (F[1][0] * F[2][1] - F[1][1] * F[2][0]);
}

// G = F^{-T} = cof(F) / J
__device__ __forceinline__ void inv_transpose(const double (&F)[3][3], double J, double (&G)[3][3]) {
  const double iJ = 1.0 / J;
  G[0][0] = (F[1][1] * F[2][2] - F[1][2] * F[2][1]) * iJ;
  G[0][1] = (F[1][2] * F[2][0] - F[1][0] * F[2][2]) * iJ;
  G[0][2] = (F[1][0] * F[2][1] - F[1][1] * F[2][0]) * iJ;
  G[1][0] = (F[0][2] * F[2][1] - F[0][1] * F[2][2]) * iJ;
  G[1][1] = (F[0][0] * F[2][2] - F[0][2] * F[2][0]) * iJ;
  G[1][2] = (F[0][1] * F[2][0] - F[0][0] * F[2][1]) * iJ;
  G[2][0] = (F[0][1] * F[1][2] - F[0][2] * F[1][1]) * iJ;
  G[2][1] = (F[0][2] * F[1][0] - F[0][0] * F[1][2]) * iJ;
  G[2][2] = (F[0][0] * F[1][1] - F[0][1] * F[1][0]) * iJ;
}

template <typename T>
__device__ __forceinline__ T clamp0(T v) { return v > T(0) ? v : T(0); }

// Writes the 78 unique values of vol * B^T [dP/dF]_+ B computed in type CT.
template <typename CT, typename ET>
__device__ __forceinline__ void element_hessian(const double (&Fd)[3][3], const double (&Dmd)[3][3],
                                                double vol, double mu_d, double lam_d, double lnJ,
                                                ET* __restrict__ out, int t, int e) {
  CT F[3][3], Dm[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) { F[i][j] = (CT)Fd[i][j]; Dm[i][j] = (CT)Dmd[i][j]; }
  const CT mu = (CT)mu_d, lam = (CT)lam_d;
  CT U[3][3], s[3], V[3][3];
  svd3<CT>(F, U, s, V);
  const CT c3 = (CT)(lam_d * lnJ - mu_d);
  const CT w[3] = {CT(1) / s[0], CT(1) / s[1], CT(1) / s[2]};
  // scaling block, projected
  CT A3[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      A3[i][j] = lam * w[i] * w[j] + (i == j ? (mu - c3 * w[i] * w[i]) : CT(0));
  CT Q3[3][3];
  sym_eig3<CT>(A3, Q3, sizeof(CT) == 8 ? 6 : 5);
  const CT ev[3] = {clamp0(A3[0][0]), clamp0(A3[1][1]), clamp0(A3[2][2])};
  CT Ms[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      Ms[i][j] = Q3[i][0] * ev[0] * Q3[j][0] + Q3[i][1] * ev[1] * Q3[j][1] + Q3[i][2] * ev[2] * Q3[j][2];
  // twist / flip pairs: c1 = (lt+ + lf+)/2, c2 = (lf+ - lt+)/2, indexed by the
  // missing axis k of pair (i, j): k=0 -> (1,2), k=1 -> (0,2), k=2 -> (0,1)
  CT c1[3], c2[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const int i = k == 0 ? 1 : 0;
    const int j = k == 2 ? 1 : 2;
    const CT g = c3 * w[i] * w[j];
    const CT lt = clamp0(mu + g), lf = clamp0(mu - g);
    c1[k] = CT(0.5) * (lt + lf);
    c2[k] = CT(0.5) * (lf - lt);
  }
  // nu_k[a]
  CT nu[3][4];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    CT sum = CT(0);
#pragma unroll
    for (int a = 1; a < 4; ++a) {
      nu[k][a] = V[0][k] * Dm[a - 1][0] + V[1][k] * Dm[a - 1][1] + V[2][k] * Dm[a - 1][2];
      sum += nu[k][a];
    }
    nu[k][0] = -sum;
  }
  const CT cv = (CT)vol;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
#pragma unroll
    for (int b = a; b < 4; ++b) {
      CT K[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int ip = 0; ip < 3; ++ip) {
          CT v = Ms[i][ip] * nu[i][a] * nu[ip][b];
          if (i == ip) {
#pragma unroll
            for (int k = 0; k < 3; ++k)
              if (k != i) v += c1[3 - i - k] * nu[k][a] * nu[k][b];
          } else {
            v += c2[3 - i - ip] * nu[ip][a] * nu[i][b];
          }
          K[i][ip] = v * cv;
        }
      CT KU[3][3];  // K U^T
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int d = 0; d < 3; ++d) KU[i][d] = K[i][0] * U[d][0] + K[i][1] * U[d][1] + K[i][2] * U[d][2];
      const int off = hess_offset(a, b);
      if (a == b) {
        int idx = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = c; d < 3; ++d) {
            const CT hv = U[c][0] * KU[0][d] + U[c][1] * KU[1][d] + U[c][2] * KU[2][d];
            out[(off + idx) * t + e] = (ET)hv;
            ++idx;
          }
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const CT hv = U[c][0] * KU[0][d] + U[c][1] * KU[1][d] + U[c][2] * KU[2][d];
            out[(off + 3 * c + d) * t + e] = (ET)hv;
          }
      }
    }
  }
}

template <typename CT, typename ET>
__global__ void __launch_bounds__(128) k_eval_elements(ElemIn in, const Vec4d* __restrict__ x,
                                                       double* __restrict__ energy,
                                                       double* __restrict__ grad,
                                                       ET* __restrict__ hess) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= in.t) return;
  const int t = in.t;
  double F[3][3], Dm[3][3];
  int vid[4];
  load_tet(in, e, x, F, Dm, vid);
  const double J = det3(F);
  if (!(J > 0.0)) {
    if (energy) energy[e] = __longlong_as_double(0x7ff0000000000000LL);
#pragma unroll
    for (int k = 0; k < 12; ++k) grad[k * t + e] = 0.0;
#pragma unroll 6
    for (int k = 0; k < 78; ++k) hess[k * t + e] = (ET)0.0;
    return;
  }
  const double vol = in.vol[e], mu = in.mu[e], lam = in.lam[e];
  const double lnJ = log(J);
  double G[3][3];
  inv_transpose(F, J, G);
  if (energy) {
    double I2 = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) I2 += F[a][b] * F[a][b];
    energy[e] = vol * (0.5 * mu * (I2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
  }
  // P = mu (F - G) + lam lnJ G ; grad_j = vol P Dm^{-1}[j-1,:]^T ; grad_0 = -sum
  double P[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) P[a][b] = mu * (F[a][b] - G[a][b]) + lam * lnJ * G[a][b];
  double g0[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int j = 1; j < 4; ++j)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v = vol * (P[c][0] * Dm[j - 1][0] + P[c][1] * Dm[j - 1][1] + P[c][2] * Dm[j - 1][2]);
      grad[(3 * j + c) * t + e] = v;
      g0[c] -= v;
    }
#pragma unroll
  for (int c = 0; c < 3; ++c) grad[c * t + e] = g0[c];
  element_hessian<CT, ET>(F, Dm, vol, mu, lam, lnJ, hess, t, e);
}

// expand the 78-value layout to full [t][12][12] float64
template <typename ET>
__global__ void k_expand_hessian(int t, const ET* __restrict__ hs, double* __restrict__ out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= t) return;
  for (int a = 0; a < 4; ++a)
    for (int b = 0; b < 4; ++b)
      for (int c = 0; c < 3; ++c)
        for (int d = 0; d < 3; ++d) {
          double v;
          if (a == b) {
            const int cc = c < d ? c : d, dd = c < d ? d : c;
            const int idx = cc == 0 ? dd : (cc == 1 ? 2 + dd : 5);
            v = load_as<double>(hs[(hess_offset(a, a) + idx) * t + e]);
          } else if (a < b) {
            v = load_as<double>(hs[(hess_offset(a, b) + 3 * c + d) * t + e]);
          } else {
            v = load_as<double>(hs[(hess_offset(b, a) + 3 * d + c) * t + e]);
          }
          out[(size_t)e * 144 + (3 * a + c) * 12 + 3 * b + d] = v;
        }
}

// ---- energy of the incremental potential at x + alpha d --------------------------
struct EnergyIn {
  ElemIn el;
  int n;
  const double* __restrict__ mass;
  const uint8_t* __restrict__ pinned;
  const Vec4d* __restrict__ xtil;
  double h2, kappa, dhat, po, pn0, pn1, pn2;
  int contact;
  const Vec4d* __restrict__ xt;  // x^t, the friction lag state
  double fmu, feps;              // friction coefficient (0: none) and mollifier width
};

__device__ __forceinline__ double barrier_b(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -r * r * log(d / dhat);
}
__device__ __forceinline__ double barrier_db(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -2.0 * r * log(d / dhat) - r * r / d;
}
__device__ __forceinline__ double barrier_d2b(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -2.0 * log(d / dhat) - 4.0 * r / d + r * r / (d * d);
}

__global__ void __launch_bounds__(kBlock) k_energy(EnergyIn in, const Vec4d* __restrict__ x,
                                                   const Vec4d* __restrict__ dvec, double alpha,
                                                   GridReduce gr, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};  // energy, number of infeasible items
  const int t = in.el.t;
  if (i < t) {
    const int e = i;
    double Dm[3][3];
    Vec4d p[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int v = in.el.tets[a * t + e];
      Vec4d xv = x[v];
      const Vec4d dv = dvec[v];
      xv.x += alpha * dv.x; xv.y += alpha * dv.y; xv.z += alpha * dv.z;
      p[a] = xv;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int b = 0; b < 3; ++b) Dm[k][b] = in.el.Dminv[(3 * k + b) * t + e];
    double F[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const double d1 = a == 0 ? p[1].x - p[0].x : a == 1 ? p[1].y - p[0].y : p[1].z - p[0].z;
      const double d2 = a == 0 ? p[2].x - p[0].x : a == 1 ? p[2].y - p[0].y : p[2].z - p[0].z;
      const double d3 = a == 0 ? p[3].x - p[0].x : a == 1 ? p[3].y - p[0].y : p[3].z - p[0].z;
#pragma unroll
      for (int b = 0; b < 3; ++b) F[a][b] = d1 * Dm[0][b] + d2 * Dm[1][b] + d3 * Dm[2][b];
    }
    const double J = det3(F);
    if (J > 0.0) {
      const double lnJ = log(J);
      double I2 = 0.0;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) I2 += F[a][b] * F[a][b];
      const double mu = in.el.mu[e], lam = in.el.lam[e];
      acc[0] = in.h2 * in.el.vol[e] * (0.5 * mu * (I2 - 3.0) - mu * lnJ + 0.5 * lam * lnJ * lnJ);
    } else {
      acc[1] = 1.0;
    }
  } else if (i < t + in.n) {
    const int v = i - t;
    Vec4d xv = x[v];
    const Vec4d dv = dvec[v];
    xv.x += alpha * dv.x; xv.y += alpha * dv.y; xv.z += alpha * dv.z;
    if (!in.pinned[v]) {
      const Vec4d xt = in.xtil[v];
      const double ex = xv.x - xt.x, ey = xv.y - xt.y, ez = xv.z - xt.z;
      acc[0] = 0.5 * in.mass[v] * (ex * ex + ey * ey + ez * ez);
    }
    if (in.contact) {
      const double dist = in.pn0 * xv.x + in.pn1 * xv.y + in.pn2 * xv.z - in.po;
      if (dist <= 0.0) acc[1] = 1.0;
      else acc[0] += in.h2 * in.kappa * barrier_b(dist, in.dhat);
      if (in.fmu > 0.0) {
        // lagged friction mu lam f0(|slip|) on every vertex in contact at x^t (Dirichlet ones included:
        // their slip is zero and the term is the constant mu lam eps / 3)
        const Vec4d xtv = in.xt[v];
        const double lam = fric_lambda(in.pn0 * xtv.x + in.pn1 * xtv.y + in.pn2 * xtv.z - in.po, in.dhat,
                                       in.kappa);
        if (lam > 0.0) {
          double u[3];
          const double y = fric_slip(xv, xtv, in.pn0, in.pn1, in.pn2, u);
          acc[0] += in.h2 * in.fmu * lam * fric_f0(y, in.feps);
        }
      }
    }
  }
  if (grid_sum<2>(acc, gr, RS_ENERGY) && threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

// ---- CCD bound and norms --------------------------------------------------------------
__global__ void k_ccd(int n, const uint8_t* __restrict__ pinned, const Vec4d* __restrict__ x,
                      const Vec4d* __restrict__ d, double pn0, double pn1, double pn2, double po,
                      double* __restrict__ tmin) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double tv = 1e300;
  if (v < n && !pinned[v]) {
    const Vec4d xv = x[v], dv = d[v];
    const double nd = pn0 * dv.x + pn1 * dv.y + pn2 * dv.z;
    if (nd < 0.0) {
      const double dist = pn0 * xv.x + pn1 * xv.y + pn2 * xv.z - po;
      tv = fmax(dist, 0.0) / (-nd);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tv = fmin(tv, __shfl_xor_sync(0xffffffffu, tv, o));
  if ((threadIdx.x & 31) == 0 && tv < 1e300) atomic_min_nonneg(tmin, tv);
}

__global__ void k_norms(int n, const Vec4d* __restrict__ d, const Vec4d* __restrict__ x,
                        const Vec4d* __restrict__ xt, double* __restrict__ out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0, b = 0.0;
  if (v < n) {
    const Vec4d dv = d[v];
    a = fmax(fabs(dv.x), fmax(fabs(dv.y), fabs(dv.z)));
    const Vec4d xv = x[v], tv = xt[v];
    b = fmax(fabs(xv.x - tv.x), fmax(fabs(xv.y - tv.y), fabs(xv.z - tv.z)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(out, a);
    atomic_max_nonneg(out + 1, b);
  }
}

// ---- launchers -----------------------------------------------------------------------
static ElemIn elem_in(mls_ctx* ctx) {
  return ElemIn{ctx->t, ctx->tets, ctx->Dminv, ctx->vol, ctx->mu, ctx->lam};
}

mls_status launch_eval_elements(mls_ctx* ctx, const Vec4d* x, double* energy_out) {
  const int nb = (ctx->t + 127) / 128;
  switch (ctx->opt.precision) {
    case MLS_FP64:
      { ++ctx->launches; k_eval_elements<double, double><<<nb, 128, 0, ctx->stream>>>(
          elem_in(ctx), x, energy_out, ctx->egrad, (double*)ctx->ehess); }
      break;
    default:
      { ++ctx->launches; k_eval_elements<float, float><<<nb, 128, 0, ctx->stream>>>(
          elem_in(ctx), x, energy_out, ctx->egrad, (float*)ctx->ehess); }
      break;
  }
  return cuda_check(ctx, cudaGetLastError(), "k_eval_elements");
}

mls_status launch_expand_hessian(mls_ctx* ctx, double* hess_out) {
  const int nb = (ctx->t + kBlock - 1) / kBlock;
  if (ctx->opt.precision == MLS_FP64)
    { ++ctx->launches; k_expand_hessian<double><<<nb, kBlock, 0, ctx->stream>>>(ctx->t, (const double*)ctx->ehess, hess_out); }
  else
    { ++ctx->launches; k_expand_hessian<float><<<nb, kBlock, 0, ctx->stream>>>(ctx->t, (const float*)ctx->ehess, hess_out); }
  return cuda_check(ctx, cudaGetLastError(), "k_expand_hessian");
}

mls_status launch_energy(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, double* E,
                         int* infeasible) {
  EnergyIn in{elem_in(ctx), ctx->n, ctx->mass, ctx->pinned, ctx->xtil, ctx->h * ctx->h,
              ctx->kappa, ctx->dhat, ctx->po, ctx->pn[0], ctx->pn[1], ctx->pn[2], ctx->contact,
              ctx->xt, ctx->contact ? ctx->fric_mu : 0.0, ctx->fric_eps_v * ctx->h_step};
  const int total = ctx->t + ctx->n;
  const int nb = (total + kBlock - 1) / kBlock;
  if (nb > kMaxPartials) return fail(ctx, MLS_EINVAL, "mesh too large for one reduction grid");
  { ++ctx->launches; k_energy<<<nb, kBlock, 0, ctx->stream>>>(in, x, d, alpha, ctx->red, ctx->dscal); }
  mls_status st = cuda_check(ctx, cudaGetLastError(), "k_energy");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host, ctx->dscal, 2 * sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream), "energy readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "energy sync");
  if (st != MLS_OK) return st;
  *E = ctx->dscal_host[0];
  *infeasible = ctx->dscal_host[1] > 0.5 ? 1 : 0;
  if (ctx->cs.on) {  // mesh-mesh pairs over the candidates of x -> x + d
    double Ec = 0.0;
    int ic = 0;
    if ((st = contact_energy(ctx, x, d, alpha, &Ec, &ic)) != MLS_OK) return st;
    *E += Ec;
    *infeasible |= ic;
  }
  return MLS_OK;
}

// Largest step fraction the CCD filter allows (Sec. 3.9): for the plane,
// 0.9 of the fraction at which the first vertex reaches it; with bodies,
// also the mesh-mesh conservative advancement (contact.cu)
mls_status launch_ccd(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double* alpha) {
  double tm = 1.0;
  if (ctx->cs.on) {
    mls_status st = contact_ccd(ctx, x, d, &tm);
    if (st != MLS_OK) return st;
  }
  if (!ctx->contact) { *alpha = tm; return MLS_OK; }
  const double big = 1e300;
  mls_status st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal + 4, &big, sizeof(double),
                                                  cudaMemcpyHostToDevice, ctx->stream), "ccd init");
  if (st != MLS_OK) return st;
  const int nb = (ctx->n + kBlock - 1) / kBlock;
  { ++ctx->launches; k_ccd<<<nb, kBlock, 0, ctx->stream>>>(ctx->n, ctx->pinned, x, d, ctx->pn[0], ctx->pn[1], ctx->pn[2],
                                        ctx->po, ctx->dscal + 4); }
  st = cuda_check(ctx, cudaGetLastError(), "k_ccd");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 4, ctx->dscal + 4, sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream), "ccd readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "ccd sync");
  if (st != MLS_OK) return st;
  const double tmin = ctx->dscal_host[4];
  *alpha = fmin(tmin >= 1e299 ? 1.0 : fmin(1.0, 0.9 * tmin), tm);
  return MLS_OK;
}

mls_status launch_norms(mls_ctx* ctx, const Vec4d* d, double* dinf, double* xdisp_inf) {
  mls_status st = cuda_check(ctx, cudaMemsetAsync(ctx->dscal + 6, 0, 2 * sizeof(double), ctx->stream),
                             "norms init");
  if (st != MLS_OK) return st;
  const int nb = (ctx->n + kBlock - 1) / kBlock;
  { ++ctx->launches; k_norms<<<nb, kBlock, 0, ctx->stream>>>(ctx->n, d, ctx->xk, ctx->xt, ctx->dscal + 6); }
  st = cuda_check(ctx, cudaGetLastError(), "k_norms");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 6, ctx->dscal + 6, 2 * sizeof(double),
                                       cudaMemcpyDeviceToHost, ctx->stream), "norms readback");
  if (st != MLS_OK) return st;
  st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "norms sync");
  if (st != MLS_OK) return st;
  *dinf = ctx->dscal_host[6];
  *xdisp_inf = ctx->dscal_host[7];
  return MLS_OK;
}

}  // namespace mls
