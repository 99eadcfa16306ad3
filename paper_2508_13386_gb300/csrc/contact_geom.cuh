// Mesh-mesh contact geometry on the device: closest points of primitive
// pairs, the closest feature, and the distance with its gradient and Hessian
// (Eq. IP term B, Sec. 3.1, which takes IPC's barrier on point-triangle and
// edge-edge pairs without writing it out); and the lagged frame, slip and
// Hessian block of the friction term D between bodies.
//
// A pair is four vertices: (p, a, b, c) for a point and a triangle, (p0, p1,
// q0, q1) for two edges.  Its distance is the Euclidean distance of the
// closest points of the closed primitives.  Where that distance is smooth it
// is the distance to the closest feature, one of
//   point-point   f = |e|^2,                     e = p - q
//   point-line    f = |e x d|^2 / |d|^2,         e = p - a, d = b - a
//   point-plane   f = (e . (e1 x e2))^2 / |e1 x e2|^2 with e = p - a, e1 = b - a,
//                 e2 = c - a, and line-line the same form with e = q0 - p0,
//                 e1 = p1 - p0, e2 = q1 - q0,
// each written in the squared distance f; the derivatives of d = sqrt(f)
// follow from those of f (grad d = grad f / 2d, Hess d = Hess f / 2d -
// grad f grad f^T / 4 d^3).  The derivatives of f are taken in the edge
// vectors and mapped to the vertices through the constant matrix C of
// those differences (grad_x = C^T grad_y, Hess_x = C^T Hess_y C).
#pragma once

#include <cmath>

namespace mls {
namespace cgeom {

struct D3 { double x, y, z; };
__host__ __device__ __forceinline__ D3 add(D3 a, D3 b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__host__ __device__ __forceinline__ D3 sub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__host__ __device__ __forceinline__ D3 scl(double s, D3 a) { return D3{s * a.x, s * a.y, s * a.z}; }
__host__ __device__ __forceinline__ double dot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ __forceinline__ D3 cross(D3 a, D3 b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__host__ __device__ __forceinline__ double comp(D3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

// closest point to p on the closed segment ab: the clamped projection
__device__ __forceinline__ D3 seg_closest(D3 p, D3 a, D3 b) {
  const D3 d = sub(b, a);
  const double L = dot(d, d);
  if (L <= 0.0) return a;
  const double t = fmin(fmax(dot(sub(p, a), d) / L, 0.0), 1.0);
  return add(a, scl(t, d));
}

// parameter of a point y of the segment ab, clamped to [0, 1]
__device__ __forceinline__ double seg_weight(D3 y, D3 a, D3 b) {
  const D3 d = sub(b, a);
  const double L = dot(d, d);
  return L <= 0.0 ? 0.0 : fmin(fmax(dot(sub(y, a), d) / L, 0.0), 1.0);
}

// Closest point of the closed triangle abc to p.  The projection on the
// triangle's plane when its barycentric coordinates (signed sub-triangle
// areas) are all non-negative; otherwise the nearest of the clamped
// projections on the edges ab, bc, ca (the first of equals).  Returns the
// squared distance; w receives the barycentric weights of the closest point.
__device__ __forceinline__ double pt_closest(D3 p, D3 a, D3 b, D3 c, double (&w)[3]) {
  const D3 n = cross(sub(b, a), sub(c, a));
  const double nn = dot(n, n);
  if (nn > 0.0) {
    const D3 q = sub(p, scl(dot(sub(p, a), n) / nn, n));
    const double wa = dot(cross(sub(b, q), sub(c, q)), n) / nn;
    const double wb = dot(cross(sub(c, q), sub(a, q)), n) / nn;
    const double wc = 1.0 - wa - wb;
    if (wa >= 0.0 && wb >= 0.0 && wc >= 0.0) {
      w[0] = wa; w[1] = wb; w[2] = wc;
      const D3 r = sub(p, q);
      return dot(r, r);
    }
  }
  const D3 s0[3] = {a, b, c}, s1[3] = {b, c, a};
  double best = INFINITY;
  w[0] = 1.0; w[1] = 0.0; w[2] = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double t = seg_weight(p, s0[k], s1[k]);
    const D3 y = add(s0[k], scl(t, sub(s1[k], s0[k])));
    const D3 r = sub(p, y);
    const double d2 = dot(r, r);
    if (d2 < best) {
      best = d2;
      w[k] = 1.0 - t;
      w[(k + 1) % 3] = t;
      w[(k + 2) % 3] = 0.0;
    }
  }
  return best;
}

// Closest points y (on p0p1) and z (on q0q1) of two closed segments: the
// minimum of |p0 + s d1 - q0 - t d2|^2 over the unit square, among the
// interior stationary point (when the 2 x 2 normal equations are regular and
// it lies in the square) and the optima on the square's four sides, in that
// order (the first of equals).  Returns the squared distance.
__device__ __forceinline__ double ee_closest(D3 p0, D3 p1, D3 q0, D3 q1, D3& y, D3& z) {
  const D3 d1 = sub(p1, p0), d2 = sub(q1, q0), r = sub(q0, p0);
  const double a00 = dot(d1, d1), a01 = -dot(d1, d2), a11 = dot(d2, d2);
  const double b0 = dot(r, d1), b1 = -dot(r, d2);
  const double det = a00 * a11 - a01 * a01;
  const double amax = fmax(fabs(a00), fmax(fabs(a01), fabs(a11)));
  double best = INFINITY;
  y = p0;
  z = q0;
  if (fabs(det) > 1e-14 * fmax(amax * amax, 1e-300)) {
    const double s = (b0 * a11 - a01 * b1) / det;
    const double t = (a00 * b1 - a01 * b0) / det;
    if (s >= 0.0 && s <= 1.0 && t >= 0.0 && t <= 1.0) {
      y = add(p0, scl(s, d1));
      z = add(q0, scl(t, d2));
      const D3 e = sub(y, z);
      best = dot(e, e);
    }
  }
  const D3 ends[4] = {p0, p1, q0, q1};
  for (int k = 0; k < 4; ++k) {
    D3 yy, zz;
    if (k < 2) { yy = ends[k]; zz = seg_closest(yy, q0, q1); }
    else { zz = ends[k]; yy = seg_closest(zz, p0, p1); }
    const D3 e = sub(yy, zz);
    const double d2v = dot(e, e);
    if (d2v < best) { best = d2v; y = yy; z = zz; }
  }
  return best;
}

// The closest feature of a pair: `form` 0 point-point, 1 point-line,
// 2 point-plane, 3 line-line; nv of the pair's four vertices (local indices
// idx) take part.  Weights within 1e-12 of an end count as that end.
struct Feature {
  int form, nv;
  int idx[4];
};

__device__ __forceinline__ Feature pt_feature(D3 p, D3 a, D3 b, D3 c) {
  double w[3];
  pt_closest(p, a, b, c, w);
  int nz = 0;
  bool zero[3];
  for (int k = 0; k < 3; ++k) { zero[k] = fabs(w[k]) <= 1e-12; nz += zero[k]; }
  Feature f{};
  if (nz == 0) {
    f.form = 2; f.nv = 4;
    f.idx[0] = 0; f.idx[1] = 1; f.idx[2] = 2; f.idx[3] = 3;
  } else if (nz == 1) {
    f.form = 1; f.nv = 3; f.idx[0] = 0;
    int q = 1;
    for (int k = 0; k < 3; ++k)
      if (!zero[k]) f.idx[q++] = 1 + k;
  } else {
    int am = 0;
    for (int k = 1; k < 3; ++k)
      if (w[k] > w[am]) am = k;
    f.form = 0; f.nv = 2; f.idx[0] = 0; f.idx[1] = 1 + am;
  }
  return f;
}

__device__ __forceinline__ Feature ee_feature(D3 p0, D3 p1, D3 q0, D3 q1) {
  D3 y, z;
  ee_closest(p0, p1, q0, q1, y, z);
  const double s = seg_weight(y, p0, p1), t = seg_weight(z, q0, q1);
  const bool s_end = s <= 1e-12 || s >= 1.0 - 1e-12;
  const bool t_end = t <= 1e-12 || t >= 1.0 - 1e-12;
  Feature f{};
  if (!s_end && !t_end) {
    f.form = 3; f.nv = 4;
    f.idx[0] = 0; f.idx[1] = 1; f.idx[2] = 2; f.idx[3] = 3;
  } else if (s_end && t_end) {
    f.form = 0; f.nv = 2; f.idx[0] = s < 0.5 ? 0 : 1; f.idx[1] = t < 0.5 ? 2 : 3;
  } else if (s_end) {
    f.form = 1; f.nv = 3; f.idx[0] = s < 0.5 ? 0 : 1; f.idx[1] = 2; f.idx[2] = 3;
  } else {
    f.form = 1; f.nv = 3; f.idx[0] = t < 0.5 ? 2 : 3; f.idx[1] = 0; f.idx[2] = 1;
  }
  return f;
}

// pair distance: point-triangle (kind 0) or edge-edge (kind 1)
__device__ __forceinline__ double pair_distance(int kind, const D3 (&P)[4]) {
  if (kind == 0) {
    double w[3];
    return sqrt(pt_closest(P[0], P[1], P[2], P[3], w));
  }
  D3 y, z;
  return sqrt(ee_closest(P[0], P[1], P[2], P[3], y, z));
}

// ---- derivatives of f = d^2 in the edge vectors -------------------------------------------
// symmetric matrices are kept whole, row-major, in arrays of (3 nb)^2

// s [v]x (the cross-product matrix of v) added into the 3 x 3 block (r0, c0)
__device__ __forceinline__ void add_skew(double* H, int ld, int r0, int c0, D3 v, double s) {
  H[(r0 + 0) * ld + c0 + 1] += -s * v.z; H[(r0 + 0) * ld + c0 + 2] += s * v.y;
  H[(r0 + 1) * ld + c0 + 0] += s * v.z;  H[(r0 + 1) * ld + c0 + 2] += -s * v.x;
  H[(r0 + 2) * ld + c0 + 0] += -s * v.y; H[(r0 + 2) * ld + c0 + 1] += s * v.x;
}
// s a b^T into block (r0, c0)
__device__ __forceinline__ void add_outer(double* H, int ld, int r0, int c0, D3 a, D3 b, double s) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[(r0 + i) * ld + c0 + j] += s * comp(a, i) * comp(b, j);
}
// s I into block (r0, c0)
__device__ __forceinline__ void add_eye(double* H, int ld, int r0, int c0, double s) {
  for (int i = 0; i < 3; ++i) H[(r0 + i) * ld + c0 + i] += s;
}

// point-plane / line-line: f = s^2 / m, s = e . n, m = n . n, n = e1 x e2;
// y = (e, e1, e2), g [9], H [81]
__device__ __forceinline__ double form_plane(D3 e, D3 e1, D3 e2, double* g, double* H) {
  const D3 n = cross(e1, e2);
  const double s = dot(e, n), m = dot(n, n);
  double gs[9], gm[9];
  const D3 a1 = cross(e2, e), a2 = cross(e, e1), b1 = cross(e2, n), b2 = cross(n, e1);
  for (int k = 0; k < 3; ++k) {
    gs[k] = comp(n, k); gs[3 + k] = comp(a1, k); gs[6 + k] = comp(a2, k);
    gm[k] = 0.0; gm[3 + k] = 2.0 * comp(b1, k); gm[6 + k] = 2.0 * comp(b2, k);
  }
  const double im = 1.0 / m, s2 = s * s;
  const double c_ss = 2.0 * im, c_hs = 2.0 * s * im, c_sm = -2.0 * s * im * im, c_hm = -s2 * im * im,
               c_mm = 2.0 * s2 * im * im * im;
  for (int i = 0; i < 9; ++i) {
    g[i] = c_hs * gs[i] - s2 * im * im * gm[i];
    for (int j = 0; j < 9; ++j)
      H[i * 9 + j] = c_ss * gs[i] * gs[j] + c_sm * (gs[i] * gm[j] + gm[i] * gs[j]) + c_mm * gm[i] * gm[j];
  }
  // + (2 s / m) Hess s: blocks (e, e1) = -[e2]x, (e, e2) = [e1]x, (e1, e2) = -[e]x and transposes
  add_skew(H, 9, 0, 3, e2, -c_hs); add_skew(H, 9, 3, 0, e2, c_hs);
  add_skew(H, 9, 0, 6, e1, c_hs);  add_skew(H, 9, 6, 0, e1, -c_hs);
  add_skew(H, 9, 3, 6, e, -c_hs);  add_skew(H, 9, 6, 3, e, c_hs);
  // - (s^2 / m^2) Hess m: (e1, e1) = 2(|e2|^2 I - e2 e2^T), (e2, e2) = 2(|e1|^2 I - e1 e1^T),
  // (e1, e2) = 2(e1 e2^T - (e1.e2) I) - 2 [n]x, (e2, e1) its transpose
  add_eye(H, 9, 3, 3, 2.0 * c_hm * dot(e2, e2)); add_outer(H, 9, 3, 3, e2, e2, -2.0 * c_hm);
  add_eye(H, 9, 6, 6, 2.0 * c_hm * dot(e1, e1)); add_outer(H, 9, 6, 6, e1, e1, -2.0 * c_hm);
  add_outer(H, 9, 3, 6, e1, e2, 2.0 * c_hm); add_eye(H, 9, 3, 6, -2.0 * c_hm * dot(e1, e2));
  add_skew(H, 9, 3, 6, n, -2.0 * c_hm);
  add_outer(H, 9, 6, 3, e2, e1, 2.0 * c_hm); add_eye(H, 9, 6, 3, -2.0 * c_hm * dot(e1, e2));
  add_skew(H, 9, 6, 3, n, 2.0 * c_hm);
  return s2 * im;
}

// point-line: f = u / w, u = |c|^2, c = e x d, w = |d|^2; y = (e, d), g [6], H [36]
__device__ __forceinline__ double form_line(D3 e, D3 d, double* g, double* H) {
  const D3 c = cross(e, d);
  const double u = dot(c, c), w = dot(d, d);
  double gu[6], gw[6];
  const D3 a1 = cross(d, c), a2 = cross(c, e);
  for (int k = 0; k < 3; ++k) {
    gu[k] = 2.0 * comp(a1, k); gu[3 + k] = 2.0 * comp(a2, k);
    gw[k] = 0.0; gw[3 + k] = 2.0 * comp(d, k);
  }
  const double iw = 1.0 / w;
  for (int i = 0; i < 6; ++i) {
    g[i] = gu[i] * iw - u * gw[i] * iw * iw;
    for (int j = 0; j < 6; ++j)
      H[i * 6 + j] = -(gu[i] * gw[j] + gw[i] * gu[j]) * iw * iw + 2.0 * u * gw[i] * gw[j] * iw * iw * iw;
  }
  // + Hess u / w: (e, e) = 2(w I - d d^T), (d, d) = 2(|e|^2 I - e e^T), (e, d) = 2(e d^T - (e.d) I) - 2 [c]x
  add_eye(H, 6, 0, 0, 2.0 * w * iw); add_outer(H, 6, 0, 0, d, d, -2.0 * iw);
  add_eye(H, 6, 3, 3, 2.0 * dot(e, e) * iw); add_outer(H, 6, 3, 3, e, e, -2.0 * iw);
  add_outer(H, 6, 0, 3, e, d, 2.0 * iw); add_eye(H, 6, 0, 3, -2.0 * dot(e, d) * iw); add_skew(H, 6, 0, 3, c, -2.0 * iw);
  add_outer(H, 6, 3, 0, d, e, 2.0 * iw); add_eye(H, 6, 3, 0, -2.0 * dot(e, d) * iw); add_skew(H, 6, 3, 0, c, 2.0 * iw);
  // - u Hess w / w^2: (d, d) = 2 I
  add_eye(H, 6, 3, 3, -2.0 * u * iw * iw);
  return u * iw;
}

// The feature's squared distance f in its nb edge vectors y: gy [3 nb],
// Hy [3 nb x 3 nb] (leading dimension 3 nb), and the map C [nb][nv] from
// the feature's vertices (local order F.idx) to the edge vectors, edge
// vector k = sum_v C[k][v] x_idx[v].  Returns f.
__device__ __forceinline__ double feature_form(const Feature& F, const D3 (&P)[4], double* gy, double* Hy,
                                               double (&C)[3][4], int& nb) {
  for (int k = 0; k < 3; ++k)
    for (int v = 0; v < 4; ++v) C[k][v] = 0.0;
  const D3 x0 = P[F.idx[0]], x1 = P[F.idx[1]];
  if (F.form == 0) {
    nb = 1;
    const D3 e = sub(x0, x1);
    for (int k = 0; k < 3; ++k) gy[k] = 2.0 * comp(e, k);
    for (int k = 0; k < 9; ++k) Hy[k] = (k % 4 == 0) ? 2.0 : 0.0;
    C[0][0] = 1; C[0][1] = -1;
    return dot(e, e);
  }
  if (F.form == 1) {
    nb = 2;
    C[0][0] = 1; C[0][1] = -1;
    C[1][1] = -1; C[1][2] = 1;
    return form_line(sub(x0, x1), sub(P[F.idx[2]], x1), gy, Hy);
  }
  nb = 3;
  const D3 x2 = P[F.idx[2]], x3 = P[F.idx[3]];
  if (F.form == 2) {
    C[0][0] = 1; C[0][1] = -1;
    C[1][1] = -1; C[1][2] = 1;
    C[2][1] = -1; C[2][3] = 1;
    return form_plane(sub(x0, x1), sub(x2, x1), sub(x3, x1), gy, Hy);
  }
  C[0][0] = -1; C[0][2] = 1;
  C[1][0] = -1; C[1][1] = 1;
  C[2][2] = -1; C[2][3] = 1;
  return form_plane(sub(x2, x0), sub(x1, x0), sub(x3, x2), gy, Hy);
}

// Distance d of the pair's feature with grad d [12] and Hess d [144] over
// the pair's 12 stacked coordinates (zero outside the feature's vertices).
// Kept out of line: inlined into the pair kernel of the assembly, the
// projected Hessians came out wrong while the same code in the derivative
// test kernel was right; out of line both match the oracle.
__device__ __noinline__ double feature_derivatives(const Feature& F, const D3 (&P)[4], double* gd, double* Hd) {
  double gy[9], Hy[81], C[3][4];
  int nb;
  const double f = feature_form(F, P, gy, Hy, C, nb);
  const int ny = 3 * nb;
  const double d = sqrt(f);
  const double i2d = 0.5 / d, i4d3 = 0.25 / (d * d * d);
  for (int k = 0; k < 12; ++k) gd[k] = 0.0;
  for (int k = 0; k < 144; ++k) Hd[k] = 0.0;
  double gx[12];
  for (int v = 0; v < F.nv; ++v)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < nb; ++k) s += C[k][v] * gy[3 * k + c];
      gx[3 * v + c] = s;
    }
  for (int v = 0; v < F.nv; ++v)
    for (int c = 0; c < 3; ++c) gd[3 * F.idx[v] + c] = gx[3 * v + c] * i2d;
  for (int v = 0; v < F.nv; ++v)
    for (int w = 0; w < F.nv; ++w)
      for (int c = 0; c < 3; ++c)
        for (int e = 0; e < 3; ++e) {
          double s = 0.0;
          for (int k = 0; k < nb; ++k) {
            if (C[k][v] == 0.0) continue;
            for (int l = 0; l < nb; ++l) s += C[k][v] * C[l][w] * Hy[(3 * k + c) * ny + 3 * l + e];
          }
          Hd[(3 * F.idx[v] + c) * 12 + 3 * F.idx[w] + e] = s * i2d - gx[3 * v + c] * gx[3 * w + e] * i4d3;
        }
  return d;
}

// ---- the barrier Hessian in the edge-vector space ----------------------------------------
// Every distance formula depends on the vertices only through the feature's
// edge vectors y = (C (x) I3) x, so grad_x d = C^T grad_y d and
// Hess_x = C^T M C with M the Hessian in y (C stands for C (x) I3 here).
// With the thin QR factorisation C^T = Q R (Q [nv][nb] with orthonormal
// columns, R [nb][nb] upper triangular), Hess_x = Q (R M R^T) Q^T, so the
// nonzero eigenpairs of the 3 nv x 3 nv block come from N = R M R^T of order
// 3 nb (9, 6 or 3 rather than 12, 9 or 6), and its projection to the PSD
// cone is Q N_+ Q^T.
struct Reduced {
  int nb;
  double d;
  double gdy[9];    // grad_y d
  double Mdy[81];   // Hess_y d (leading dimension 3 nb)
  double C[3][4];   // edge-vector map
  double Q[4][3];   // thin QR factors of C^T
  double R[3][3];
};

__device__ __noinline__ void feature_reduced(const Feature& F, const D3 (&P)[4], Reduced& Rd) {
  double gy[9];
  int nb;
  const double f = feature_form(F, P, gy, Rd.Mdy, Rd.C, nb);
  Rd.nb = nb;
  const int ny = 3 * nb;
  const double d = sqrt(f);
  Rd.d = d;
  const double i2d = 0.5 / d, i4d3 = 0.25 / (d * d * d);
  for (int i = 0; i < ny; ++i) {
    Rd.gdy[i] = gy[i] * i2d;
    for (int j = 0; j < ny; ++j) Rd.Mdy[i * ny + j] = Rd.Mdy[i * ny + j] * i2d - gy[i] * gy[j] * i4d3;
  }
  // modified Gram-Schmidt on the columns of C^T (the rows of C)
  for (int k = 0; k < 3; ++k)
    for (int l = 0; l < 3; ++l) Rd.R[k][l] = 0.0;
  for (int k = 0; k < nb; ++k) {
    double q[4];
    for (int v = 0; v < 4; ++v) q[v] = v < F.nv ? Rd.C[k][v] : 0.0;
    for (int l = 0; l < k; ++l) {
      double r = 0.0;
      for (int v = 0; v < F.nv; ++v) r += Rd.Q[v][l] * q[v];
      Rd.R[l][k] = r;
      for (int v = 0; v < F.nv; ++v) q[v] -= r * Rd.Q[v][l];
    }
    double nrm = 0.0;
    for (int v = 0; v < F.nv; ++v) nrm += q[v] * q[v];
    nrm = sqrt(nrm);
    Rd.R[k][k] = nrm;
    for (int v = 0; v < 4; ++v) Rd.Q[v][k] = v < F.nv ? q[v] / nrm : 0.0;
  }
}

// Entry (a, b) of N = R M R^T, M = kappa (b'' grad_y d grad_y d^T + b' Hess_y d)
// given b1 = kappa b'(d), b2 = kappa b''(d); a = 3 k + c, b = 3 l + e
__device__ __forceinline__ double reduced_entry(const Reduced& Rd, double b1, double b2, int a, int b) {
  const int ny = 3 * Rd.nb, k = a / 3, c = a % 3, l = b / 3, e = b % 3;
  double s = 0.0;
  for (int kk = k; kk < Rd.nb; ++kk)
    for (int ll = l; ll < Rd.nb; ++ll) {
      const int i = 3 * kk + c, j = 3 * ll + e;
      s += Rd.R[k][kk] * (b2 * Rd.gdy[i] * Rd.gdy[j] + b1 * Rd.Mdy[i * ny + j]) * Rd.R[l][ll];
    }
  return s;
}

// Entry ((v, c), (w, e)) of Q N_+ Q^T over the feature's vertices, N_+ [ny][ld]
__device__ __forceinline__ double reduced_back(const Reduced& Rd, const double* Np, int ld, int v, int c, int w,
                                               int e) {
  double s = 0.0;
  for (int k = 0; k < Rd.nb; ++k)
    for (int l = 0; l < Rd.nb; ++l) s += Rd.Q[v][k] * Np[(3 * k + c) * ld + 3 * l + e] * Rd.Q[w][l];
  return s;
}

// ---- friction between bodies (Eq. IP term D) ----------------------------------------------
// The ground friction with the plane replaced by the pair's closest points,
// lagged at x^t for the whole step.  The frame of a pair: the weights w with
// which its closest-point difference is y - z = sum_j w_j P_j (point-triangle:
// 1 and minus the closest point's barycentric weights; edge-edge: 1 - s, s,
// -(1 - t), -t; they sum to zero), and the unit normal n along y - z.
// Returns the distance |y - z|.
__device__ __forceinline__ double friction_frame(int kind, const D3 (&P)[4], double (&w)[4], D3& n) {
  if (kind == 0) {
    double b[3];
    pt_closest(P[0], P[1], P[2], P[3], b);
    w[0] = 1.0; w[1] = -b[0]; w[2] = -b[1]; w[3] = -b[2];
  } else {
    D3 y, z;
    ee_closest(P[0], P[1], P[2], P[3], y, z);
    const double s = seg_weight(y, P[0], P[1]), t = seg_weight(z, P[2], P[3]);
    w[0] = 1.0 - s; w[1] = s; w[2] = -(1.0 - t); w[3] = -t;
  }
  D3 e{0.0, 0.0, 0.0};
  for (int j = 0; j < 4; ++j) e = add(e, scl(w[j], P[j]));
  const double d = sqrt(dot(e, e));
  n = d > 0.0 ? scl(1.0 / d, e) : D3{0.0, 0.0, 0.0};
  return d;
}

// The slip of a lagged pair over the step, u = (I - n n^T) sum_j w_j dx_j
// with dx_j = x_j - x_j^t; returns |u|.
__device__ __forceinline__ double friction_slip(const double (&w)[4], D3 n, const D3 (&dx)[4], D3& u) {
  D3 r{0.0, 0.0, 0.0};
  for (int j = 0; j < 4; ++j) r = add(r, scl(w[j], dx[j]));
  u = sub(r, scl(dot(r, n), n));
  return sqrt(dot(u, u));
}

// The 3 x 3 K of the pair's Hessian, d2D/dx_i dx_j = w_i w_j mu lambda K:
// K = ratio (I - n n^T) + (slope - ratio) u^ u^T with ratio = f1(y)/y,
// slope = f1'(y), u^ = u / y (at y = 0 both factors are 2/eps and u^ drops
// out).  Positive semi-definite since ratio > 0 and slope >= 0.
__device__ __forceinline__ void friction_block(D3 n, D3 u, double y, double ratio, double slope, double (&K)[9]) {
  const double nn[3] = {n.x, n.y, n.z};
  const double uh[3] = {y > 0.0 ? u.x / y : 0.0, y > 0.0 ? u.y / y : 0.0, y > 0.0 ? u.z / y : 0.0};
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      K[3 * r + c] = ratio * ((r == c ? 1.0 : 0.0) - nn[r] * nn[c]) + (slope - ratio) * uh[r] * uh[c];
}

}  // namespace cgeom
}  // namespace mls
