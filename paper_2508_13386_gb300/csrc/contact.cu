// Mesh-mesh contact on the GPU: the barrier term B of Eq. IP between the
// surface primitives of different bodies (Sec. 3.1, which takes IPC's
// barrier without writing it out) and the CCD filter of the line search
// (Sec. 3.9, additive CCD).
//
//   pairs      point-triangle (surface vertex, boundary face) and edge-edge
//              (boundary edges) pairs of different bodies
//   broad      a hashed uniform grid: every face and edge is entered, with its
//              box grown by dhat, in each cell the box meets; each surface
//              vertex and edge walks the cells its own box meets.  A pair is
//              kept in the one cell that holds the lower corner of the two
//              boxes' intersection, so it is found once.  At an assembly
//              iterate the pairs are filtered to distance < dhat; for a line
//              search the boxes cover the whole segment x -> x + d, so every
//              pair that comes within dhat anywhere on it is a candidate
//   barrier    kappa b(d) per pair with its gradient and its 12 x 12 Hessian
//              kappa (b'' grad d grad d^T + b' Hess d) projected to the PSD
//              cone (contact_geom.cuh)
//   H          each pair adds its 3 x 3 vertex blocks (i, j); blocks between
//              vertices of one body land in H's element pattern, blocks
//              between bodies in spare slots that every surface-vertex row
//              keeps after its element blocks and claims per assembly
//   coarse     the cross-body blocks add U_i^T H_ij U_j to U^T H U (the
//              element pattern's blocks are in H's values already)
//   CCD        conservative advancement per candidate: from distance d at t,
//              t += (d - s d0) / L with L the additive bound (the two
//              primitives' largest vertex displacements relative to the
//              pair's mean displacement), s = 0.1; the step fraction is the
//              smallest over the candidates
#include <algorithm>
#include <array>
#include <cstring>

#include "contact_geom.cuh"
#include "mls_internal.cuh"

namespace mls {

using cgeom::D3;

// device counters
enum { kCntEnt = 0, kCntPT, kCntEE, kCntFlags, kCntXc, kCntWords = 8 };
// flags
enum { kFlagSlots = 1, kFlagSpan = 2, kFlagTable = 4, kFlagRange = 8 };
constexpr int kMaxCellsPerBox = 4096;   // a larger box asks for a coarser grid
constexpr unsigned long long kEmptyKey = ~0ull;
constexpr double kCcdS = 0.1;           // CCD keeps every pair at >= s of its distance
constexpr int kCcdMaxIter = 100000;
constexpr double kCcdRtol = 1e-10;

__device__ __forceinline__ D3 pos(const Vec4d* __restrict__ x, const Vec4d* __restrict__ d, double alpha, int v) {
  const Vec4d p = x[v];
  if (!d) return D3{p.x, p.y, p.z};
  const Vec4d q = d[v];
  return D3{p.x + alpha * q.x, p.y + alpha * q.y, p.z + alpha * q.z};
}

struct Box { double lo[3], hi[3]; };

// box of the vertices vs[0..k) over the segment x -> x + d (d nullable), grown by pad
__device__ __forceinline__ Box prim_box(const Vec4d* __restrict__ x, const Vec4d* __restrict__ d, const int* vs,
                                        int k, double pad) {
  Box b;
  for (int c = 0; c < 3; ++c) { b.lo[c] = INFINITY; b.hi[c] = -INFINITY; }
  for (int i = 0; i < k; ++i) {
    const D3 p = pos(x, nullptr, 0.0, vs[i]);
    for (int c = 0; c < 3; ++c) {
      b.lo[c] = fmin(b.lo[c], cgeom::comp(p, c));
      b.hi[c] = fmax(b.hi[c], cgeom::comp(p, c));
    }
    if (d) {
      const D3 q = pos(x, d, 1.0, vs[i]);
      for (int c = 0; c < 3; ++c) {
        b.lo[c] = fmin(b.lo[c], cgeom::comp(q, c));
        b.hi[c] = fmax(b.hi[c], cgeom::comp(q, c));
      }
    }
  }
  for (int c = 0; c < 3; ++c) { b.lo[c] -= pad; b.hi[c] += pad; }
  return b;
}

__device__ __forceinline__ uint32_t cell_hash(int ix, int iy, int iz) {
  return ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^ ((uint32_t)iz * 83492791u);
}

// cells are addressed by 21-bit coordinates, |i| < 2^20
constexpr double kCellRange = 1048000.0;
__device__ __forceinline__ unsigned long long cell_key(int ix, int iy, int iz) {
  return (unsigned long long)(ix + (1 << 20)) | ((unsigned long long)(iy + (1 << 20)) << 21) |
         ((unsigned long long)(iz + (1 << 20)) << 42);
}

// integer cell range of a box; false (and a flag) when it is out of range or too large
__device__ __forceinline__ bool cell_range(const Box& b, double inv_cell, int (&c0)[3], int (&c1)[3], int* flags) {
  int64_t count = 1;
  for (int c = 0; c < 3; ++c) {
    const double l = floor(b.lo[c] * inv_cell), h = floor(b.hi[c] * inv_cell);
    if (!(l > -kCellRange && h < kCellRange)) {
      atomicOr(flags, kFlagRange);
      return false;
    }
    c0[c] = (int)l;
    c1[c] = (int)h;
    count *= (int64_t)(c1[c] - c0[c] + 1);
  }
  if (count > kMaxCellsPerBox) {
    atomicOr(flags, kFlagSpan);
    return false;
  }
  return true;
}

// monotone map of doubles to unsigned 64-bit keys (for atomic min / max)
__device__ __forceinline__ unsigned long long dkey(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  return __longlong_as_double((long long)((k >> 63) ? (k & 0x7fffffffffffffffull) : ~k));
}

constexpr int kMaxBodyBoxes = 64;  // bodies up to this count get the box prefilter

// per-body boxes of the surface vertices over x -> x + d: block-level
// reduction in shared memory, one global atomic per block and coordinate
__global__ void __launch_bounds__(kBlock) k_body_boxes(const int2* __restrict__ sverts, int nsv, int nbody,
                                                       const Vec4d* __restrict__ x, const Vec4d* __restrict__ d,
                                                       unsigned long long* __restrict__ lo,
                                                       unsigned long long* __restrict__ hi) {
  __shared__ unsigned long long slo[kMaxBodyBoxes * 3], shi[kMaxBodyBoxes * 3];
  for (int k = threadIdx.x; k < 3 * nbody; k += blockDim.x) {
    slo[k] = ~0ull;
    shi[k] = 0ull;
  }
  __syncthreads();
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nsv) {
    const int2 sv = sverts[q];
    for (int pass = 0; pass < (d ? 2 : 1); ++pass) {
      const D3 p = pos(x, d, pass ? 1.0 : 0.0, sv.x);
      for (int c = 0; c < 3; ++c) {
        const unsigned long long k = dkey(cgeom::comp(p, c));
        atomicMin(slo + 3 * sv.y + c, k);
        atomicMax(shi + 3 * sv.y + c, k);
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 3 * nbody; k += blockDim.x) {
    if (slo[k] != ~0ull) atomicMin(lo + k, slo[k]);
    if (shi[k] != 0ull) atomicMax(hi + k, shi[k]);
  }
}

struct GridView {
  int nf, ne, nsv, nbody;
  const int4* __restrict__ faces;
  const int4* __restrict__ edges;
  const int2* __restrict__ sverts;
  int* head;                 // [2 << hbits]: faces' buckets, then edges'
  int hmask;
  int4* ent;                 // {primitive, body, cell key low, cell key high}
  int* next;
  int64_t ecap;
  double* boxes;
  int* cnt;
  const unsigned long long* blo;  // per-body boxes (nullable: no prefilter)
  const unsigned long long* bhi;
  double inv_cell, dhat;
};

// enter every face and edge (box grown by dhat) into the cells its box meets
__global__ void k_grid_insert(GridView G, const Vec4d* __restrict__ x, const Vec4d* __restrict__ d) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= G.nf + G.ne) return;
  int vs[3], k, body;
  if (p < G.nf) {
    const int4 f = G.faces[p];
    vs[0] = f.x; vs[1] = f.y; vs[2] = f.z; k = 3; body = f.w;
  } else {
    const int4 e = G.edges[p - G.nf];
    vs[0] = e.x; vs[1] = e.y; vs[2] = e.y; k = 2; body = e.z;
  }
  const Box b = prim_box(x, d, vs, k, G.dhat);
  for (int c = 0; c < 3; ++c) {
    G.boxes[6 * (int64_t)p + c] = b.lo[c];
    G.boxes[6 * (int64_t)p + 3 + c] = b.hi[c];
  }
  int c0[3], c1[3];
  if (!cell_range(b, G.inv_cell, c0, c1, G.cnt + kCntFlags)) return;
  int* head = G.head + (p < G.nf ? 0 : G.hmask + 1);
  for (int iz = c0[2]; iz <= c1[2]; ++iz)
    for (int iy = c0[1]; iy <= c1[1]; ++iy)
      for (int ix = c0[0]; ix <= c1[0]; ++ix) {
        const int e = atomicAdd(G.cnt + kCntEnt, 1);
        if (e >= G.ecap) continue;  // counted; the host grows the table and enters again
        const unsigned long long key = cell_key(ix, iy, iz);
        G.ent[e] = make_int4(p, body, (int)(unsigned)key, (int)(unsigned)(key >> 32));
        G.next[e] = atomicExch(head + (cell_hash(ix, iy, iz) & G.hmask), e);
      }
}

struct PairOut {
  int2* pt;
  int2* ee;
  int64_t cap;
};

// Each surface vertex (point-triangle, against the faces' buckets) and edge
// (edge-edge, the edges' buckets, partner index above its own) walks the
// cells of its own box; primitives whose box meets no other body's box are
// skipped.  Proximity mode (d null): keep pairs at distance < dhat at x.
// Sweep mode: keep every candidate.
__global__ void k_grid_query(GridView G, const Vec4d* __restrict__ x, const Vec4d* __restrict__ d, PairOut out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= G.nsv + G.ne) return;
  const bool is_pt = q < G.nsv;
  int vs[2], k, body, self;
  if (is_pt) {
    const int2 s = G.sverts[q];
    vs[0] = s.x; vs[1] = s.x; k = 1; body = s.y; self = s.x;
  } else {
    const int4 e = G.edges[q - G.nsv];
    vs[0] = e.x; vs[1] = e.y; k = 2; body = e.z; self = q - G.nsv;
  }
  const Box b = prim_box(x, d, vs, k, 0.0);
  if (G.blo) {  // near another body at all?
    bool near = false;
    for (int o = 0; o < G.nbody && !near; ++o) {
      if (o == body) continue;
      bool m = true;
      for (int c = 0; c < 3; ++c)
        m = m && b.hi[c] >= dkey_inv(G.blo[3 * o + c]) - 2.0 * G.dhat &&
            b.lo[c] <= dkey_inv(G.bhi[3 * o + c]) + 2.0 * G.dhat;
      near = m;
    }
    if (!near) return;
  }
  int c0[3], c1[3];
  if (!cell_range(b, G.inv_cell, c0, c1, G.cnt + kCntFlags)) return;
  const double dh = G.dhat;
  const int* head = G.head + (is_pt ? 0 : G.hmask + 1);
  for (int iz = c0[2]; iz <= c1[2]; ++iz)
    for (int iy = c0[1]; iy <= c1[1]; ++iy)
      for (int ix = c0[0]; ix <= c1[0]; ++ix) {
        const unsigned long long key = cell_key(ix, iy, iz);
        const int klo = (int)(unsigned)key, khi = (int)(unsigned)(key >> 32);
        int e = __ldcg(head + (cell_hash(ix, iy, iz) & G.hmask));
        while (e >= 0) {
          const int4 en = G.ent[e];
          e = G.next[e];
          if (en.z != klo || en.w != khi || en.y == body) continue;
          const int p = en.x;
          const int other = is_pt ? p : p - G.nf;
          if (!is_pt && other <= self) continue;
          // boxes meet, and this cell holds the lower corner of their intersection
          const double* ib = G.boxes + 6 * (int64_t)p;
          bool meet = true, own = true;
          const int cc[3] = {ix, iy, iz};
          for (int c = 0; c < 3; ++c) {
            const double lo = fmax(b.lo[c], ib[c]), hi = fmin(b.hi[c], ib[3 + c]);
            if (lo > hi) meet = false;
            if ((int)floor(lo * G.inv_cell) != cc[c]) own = false;
          }
          if (!meet || !own) continue;
          if (!d) {  // proximity: the exact distance decides
            D3 P[4];
            if (is_pt) {
              const int4 f = G.faces[p];
              P[0] = pos(x, nullptr, 0.0, self); P[1] = pos(x, nullptr, 0.0, f.x);
              P[2] = pos(x, nullptr, 0.0, f.y); P[3] = pos(x, nullptr, 0.0, f.z);
            } else {
              const int4 ej = G.edges[other];
              P[0] = pos(x, nullptr, 0.0, vs[0]); P[1] = pos(x, nullptr, 0.0, vs[1]);
              P[2] = pos(x, nullptr, 0.0, ej.x); P[3] = pos(x, nullptr, 0.0, ej.y);
            }
            if (!(cgeom::pair_distance(is_pt ? 0 : 1, P) < dh)) continue;
          }
          const int slot = atomicAdd(G.cnt + (is_pt ? kCntPT : kCntEE), 1);
          if (slot < out.cap) {
            if (is_pt) out.pt[slot] = make_int2(self, other);
            else out.ee[slot] = make_int2(self, other);
          }
        }
      }
}

__device__ __forceinline__ void pair_vertices(int kind, int2 pr, const int4* __restrict__ faces,
                                              const int4* __restrict__ edges, int (&v)[4]) {
  if (kind == 0) {
    const int4 f = faces[pr.y];
    v[0] = pr.x; v[1] = f.x; v[2] = f.y; v[3] = f.z;
  } else {
    const int4 a = edges[pr.x], b = edges[pr.y];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}

__device__ __forceinline__ double bar_b(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -r * r * log(d / dhat);
}
__device__ __forceinline__ double bar_b1(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -2.0 * r * log(d / dhat) - r * r / d;
}
__device__ __forceinline__ double bar_b2(double d, double dhat) {
  if (d >= dhat) return 0.0;
  const double r = d - dhat;
  return -2.0 * log(d / dhat) - 4.0 * r / d + r * r / (d * d);
}

struct CouplingView {
  unsigned long long* key;
  double* val;
  int mask;
  int* flags;
};

__device__ __forceinline__ int coupling_slot(const CouplingView& C, int i, int j) {
  const unsigned long long k = ((unsigned long long)(unsigned)i << 32) | (unsigned)j;
  const unsigned long long h = k * 0x9E3779B97F4A7C15ull;
  int s = (int)(h >> 33) & C.mask;
  for (int probe = 0; probe <= C.mask; ++probe) {
    const unsigned long long old = atomicCAS(C.key + s, kEmptyKey, k);
    if (old == kEmptyKey || old == k) return s;
    s = (s + 1) & C.mask;
  }
  atomicOr(C.flags, kFlagTable);
  return -1;
}

// ---- one warp per pair: derivatives by one lane, PSD projection by the warp ----------------
// The float64 work of a pair is too long and serial for one thread (float64
// instructions issue at a small fraction of the integer rate here), so a
// warp evaluates each pair.  Lane 0 finds the closest feature and the
// distance's derivatives in the feature's edge vectors with the thin QR
// factors of their map (contact_geom.cuh, feature_reduced); the warp forms
// the barrier Hessian's reduced matrix N = R M R^T (order 3 nb: 9, 6 or 3)
// and diagonalises it by parallel cyclic Jacobi (Golub and Van Loan,
// Sec. 8.5): in each round the index pairs of a round-robin tournament are
// rotated at once (the rotations are disjoint, so J^T A J takes one column
// pass and one row pass), n - 1 rounds a sweep, until the off-diagonal mass
// is below 1e-24 of the diagonal's; then Q N_+ Q^T is the projected 12 x 12
// pair Hessian.
constexpr int kPairWarps = 4;

struct PairWarp {
  double A[144];   // N being diagonalised (leading dimension 12), then the projected pair Hessian
  double V[144];   // N's eigenvectors
  double H[144];   // N_+
  double gx[12];   // barrier gradient over the pair's 12 coordinates
  double lam[12];  // N's eigenvalues clamped at zero
  double c[6], s[6];
  int p[6], q[6];
  double b1, b2;
  int ok, k;
  cgeom::Feature F;
  cgeom::Reduced Rd;
};

// lane 0: distance, feature and reduced derivatives of the pair P; the warp:
// the projected barrier Hessian into W.A (12 x 12, zero outside the
// feature) and the barrier gradient into W.gx.  Returns false (uniformly)
// when the pair is at or beyond dhat.  With hd_out / gd_out (testing), lane
// 0 also writes grad d and Hess d over the 12 coordinates there.
__device__ bool pair_eval_warp(int kind, const D3 (&P)[4], double kappa, double dhat, PairWarp& W, int lane,
                               double* hd_out, double* gd_out) {
  if (lane == 0) {
    const double dist = cgeom::pair_distance(kind, P);
    W.ok = (dist < dhat && dist > 0.0) || hd_out;
    if (W.ok) {
      W.F = kind == 0 ? cgeom::pt_feature(P[0], P[1], P[2], P[3]) : cgeom::ee_feature(P[0], P[1], P[2], P[3]);
      cgeom::feature_reduced(W.F, P, W.Rd);
      const double d = W.Rd.d;
      W.b1 = kappa * bar_b1(d, dhat);
      W.b2 = kappa * bar_b2(d, dhat);
      W.k = 3 * W.Rd.nb;
      for (int q = 0; q < 12; ++q) W.gx[q] = 0.0;
      for (int v = 0; v < W.F.nv; ++v)
        for (int c = 0; c < 3; ++c) {
          double sum = 0.0;
          for (int k = 0; k < W.Rd.nb; ++k) sum += W.Rd.C[k][v] * W.Rd.gdy[3 * k + c];
          W.gx[3 * W.F.idx[v] + c] = W.b1 * sum;
        }
      if (hd_out) cgeom::feature_derivatives(W.F, P, gd_out, hd_out);
    }
  }
  __syncwarp();
  if (!W.ok) return false;
  const int k = W.k;
  const cgeom::Feature F = W.F;
  for (int t = lane; t < k * k; t += 32) {
    const int a = t / k, b = t % k;
    W.A[a * 12 + b] = cgeom::reduced_entry(W.Rd, W.b1, W.b2, a, b);
    W.V[a * 12 + b] = a == b ? 1.0 : 0.0;
  }
  __syncwarp();
  const int n = k + (k & 1);  // even order of the tournament (index k stands out when k is odd)
  const int half = n / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, dia = 0.0;
    for (int t = lane; t < k * k; t += 32) {
      const int a = t / k, b = t % k;
      const double v = W.A[a * 12 + b];
      if (a == b) dia += v * v;
      else if (a < b) off += v * v;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      dia += __shfl_xor_sync(0xffffffffu, dia, o);
    }
    if (off <= 1e-24 * dia || off == 0.0) break;
    for (int r = 0; r < n - 1; ++r) {
      if (lane < half) {
        int p, q;
        if (lane == 0) {
          p = r;
          q = n - 1;
        } else {
          p = (r + lane) % (n - 1);
          q = (r - lane + n - 1) % (n - 1);
        }
        if (p > q) { const int t = p; p = q; q = t; }
        double c = 1.0, sn = 0.0;
        if (q < k) {
          const double apq = W.A[p * 12 + q], app = W.A[p * 12 + p], aqq = W.A[q * 12 + q];
          if (apq != 0.0 && apq * apq > 1e-36 * fabs(app * aqq)) {
            const double tau = (aqq - app) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
        }
        W.p[lane] = p;
        W.q[lane] = q < k ? q : p;  // a pair with the standing-out index does nothing
        W.c[lane] = c;
        W.s[lane] = sn;
      }
      __syncwarp();
      for (int t = lane; t < half * k; t += 32) {  // A <- A J and V <- V J (columns p, q)
        const int m = t / k, row = t % k;
        const int p = W.p[m], q = W.q[m];
        if (p == q) continue;
        const double c = W.c[m], sn = W.s[m];
        const double arp = W.A[row * 12 + p], arq = W.A[row * 12 + q];
        W.A[row * 12 + p] = c * arp - sn * arq;
        W.A[row * 12 + q] = sn * arp + c * arq;
        const double vrp = W.V[row * 12 + p], vrq = W.V[row * 12 + q];
        W.V[row * 12 + p] = c * vrp - sn * vrq;
        W.V[row * 12 + q] = sn * vrp + c * vrq;
      }
      __syncwarp();
      for (int t = lane; t < half * k; t += 32) {  // A <- J^T A (rows p, q)
        const int m = t / k, col = t % k;
        const int p = W.p[m], q = W.q[m];
        if (p == q) continue;
        const double c = W.c[m], sn = W.s[m];
        const double apr = W.A[p * 12 + col], aqr = W.A[q * 12 + col];
        W.A[p * 12 + col] = c * apr - sn * aqr;
        W.A[q * 12 + col] = sn * apr + c * aqr;
      }
      __syncwarp();
    }
  }
  if (lane < k) W.lam[lane] = fmax(W.A[lane * 12 + lane], 0.0);
  __syncwarp();
  for (int t = lane; t < k * k; t += 32) {  // N_+ = V max(Lambda, 0) V^T
    const int a = t / k, b = t % k;
    double sum = 0.0;
    for (int m = 0; m < k; ++m) sum += W.V[a * 12 + m] * W.lam[m] * W.V[b * 12 + m];
    W.H[a * 12 + b] = sum;
  }
  for (int t = lane; t < 144; t += 32) W.A[t] = 0.0;
  __syncwarp();
  const int kx = 3 * F.nv;
  for (int t = lane; t < kx * kx; t += 32) {  // Q N_+ Q^T on the feature's vertices
    const int a = t / kx, b = t % kx;
    W.A[(3 * F.idx[a / 3] + a % 3) * 12 + 3 * F.idx[b / 3] + b % 3] =
        cgeom::reduced_back(W.Rd, W.H, 12, a / 3, a % 3, b / 3, b % 3);
  }
  __syncwarp();
  return true;
}

// one warp per pair: the barrier gradient [12] and projected Hessian [144]
// of the pair into pg / pH (zero at or beyond dhat)
__global__ void __launch_bounds__(32 * kPairWarps) k_pair_eval(const int2* __restrict__ pt, int npt,
                                                               const int2* __restrict__ ee, int nee,
                                                               const int4* __restrict__ faces,
                                                               const int4* __restrict__ edges,
                                                               const Vec4d* __restrict__ x, double kappa,
                                                               double dhat, double* __restrict__ pg,
                                                               double* __restrict__ pH) {
  __shared__ PairWarp sw[kPairWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int idx = blockIdx.x * kPairWarps + warp;
  if (idx >= npt + nee) return;  // uniform per warp
  PairWarp& W = sw[warp];
  const int kind = idx < npt ? 0 : 1;
  int v[4];
  pair_vertices(kind, kind == 0 ? pt[idx] : ee[idx - npt], faces, edges, v);
  D3 P[4];
  for (int a = 0; a < 4; ++a) P[a] = pos(x, nullptr, 0.0, v[a]);
  double* og = pg + 12 * (int64_t)idx;
  double* oH = pH + 144 * (int64_t)idx;
  if (!pair_eval_warp(kind, P, kappa, dhat, W, lane, nullptr, nullptr)) {
    if (lane < 12) og[lane] = 0.0;
    for (int t = lane; t < 144; t += 32) oH[t] = 0.0;
    return;
  }
  if (lane < 12) og[lane] = W.gx[lane];
  for (int t = lane; t < 144; t += 32) oH[t] = W.A[t];
}

// one thread per (pair, vertex a, vertex b): block (a, b) of the pair's
// Hessian into the coupling table, and for b = 0 the gradient of vertex a
// into cgrad (Dirichlet vertices left out)
__global__ void k_pair_scatter(const int2* __restrict__ pt, int npt, const int2* __restrict__ ee, int nee,
                               const int4* __restrict__ faces, const int4* __restrict__ edges,
                               const uint8_t* __restrict__ pinned, const double* __restrict__ pg,
                               const double* __restrict__ pH, Vec4d* __restrict__ cgrad, CouplingView C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 16 * (int64_t)(npt + nee)) return;
  const int idx = (int)(t >> 4), a = (int)(t >> 2) & 3, b = (int)t & 3;
  const int kind = idx < npt ? 0 : 1;
  int v[4];
  pair_vertices(kind, kind == 0 ? pt[idx] : ee[idx - npt], faces, edges, v);
  if (pinned[v[a]] || pinned[v[b]]) return;
  if (b == 0) {
    const double* g = pg + 12 * (int64_t)idx + 3 * a;
    if (g[0] != 0.0 || g[1] != 0.0 || g[2] != 0.0) {
      atomicAdd(&cgrad[v[a]].x, g[0]);
      atomicAdd(&cgrad[v[a]].y, g[1]);
      atomicAdd(&cgrad[v[a]].z, g[2]);
    }
  }
  const double* H = pH + 144 * (int64_t)idx;
  double blk[9];
  bool nz = false;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      blk[3 * r + c] = H[(3 * a + r) * 12 + 3 * b + c];
      nz |= blk[3 * r + c] != 0.0;
    }
  if (!nz) return;
  const int s = coupling_slot(C, v[a], v[b]);
  if (s < 0) return;
  for (int q = 0; q < 9; ++q) atomicAdd(C.val + 9 * (int64_t)s + q, blk[q]);
}

// surface-vertex rows: release the spare slots claimed at the last assembly
__global__ void k_contact_reset_rows(const int2* __restrict__ sverts, int nsv, const int* __restrict__ slice_ptr,
                                     const int* __restrict__ row_len0, int* __restrict__ row_len,
                                     int* __restrict__ col) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nsv) return;
  const int i = sverts[q].x;
  const int g0 = slice_ptr[i >> 5], g1 = slice_ptr[(i >> 5) + 1], lane = i & 31;
  const int len0 = row_len0[i];
  row_len[i] = len0;
  for (int k = len0; k < g1 - g0; ++k) col[((int64_t)g0 + k) * 32 + lane] = -1;
}

template <typename T>
__device__ __forceinline__ void inv3c(const T (&A)[9], T (&R)[9]) {
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

// One thread per coupling (i, j): find its slot in row i (the diagonal, an
// element block, or a spare slot claimed by compare-and-swap), add h^2 times
// the block to the stored value, and refresh D^{-1} of row i with the
// diagonal block.  Couplings are unique, so every slot has one writer.
template <typename MT, typename VT>
__global__ void k_contact_merge(CouplingView C, const int* __restrict__ slice_ptr, const int* __restrict__ row_len0,
                                int* __restrict__ row_len, int* __restrict__ col, MT* __restrict__ val,
                                VT* __restrict__ dinv, double h2, int4* __restrict__ xc, int* __restrict__ nxc,
                                int xcap) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s > C.mask) return;
  const unsigned long long key = C.key[s];
  if (key == kEmptyKey) return;
  const int i = (int)(key >> 32), j = (int)(key & 0xffffffffu);
  const int g0 = slice_ptr[i >> 5], width = slice_ptr[(i >> 5) + 1] - g0, lane = i & 31;
  const int len0 = row_len0[i];
  int k = -1;
  bool cross = false;
  if (i == j) {
    k = 0;
  } else {
    for (int q = 1; q < len0; ++q)
      if (col[((int64_t)g0 + q) * 32 + lane] == j) { k = q; break; }
    if (k < 0) {
      for (int q = len0; q < width; ++q) {
        const int old = atomicCAS(col + ((int64_t)g0 + q) * 32 + lane, -1, j);
        if (old == -1 || old == j) {
          k = q;
          atomicMax(row_len + i, q + 1);
          cross = true;
          break;
        }
      }
    }
  }
  if (k < 0) {
    atomicOr(C.flags, kFlagSlots);
    return;
  }
  MT* out = val + ((int64_t)g0 + k) * 288 + lane;
  double blk[9];
  for (int q = 0; q < 9; ++q) {
    blk[q] = load_as<double>(out[q * 32]) + h2 * C.val[9 * (int64_t)s + q];
    out[q * 32] = from_d<MT>(blk[q]);
  }
  if (cross && xc) {
    const int e = atomicAdd(nxc, 1);
    if (e < xcap) xc[e] = make_int4(i, j, (int)(((int64_t)g0 + k) * 32 + lane), 0);
  }
  if (i == j && dinv) {
    VT A[9], R[9];
    for (int q = 0; q < 9; ++q) A[q] = load_as<VT>(from_d<MT>(blk[q]));
    inv3c<VT>(A, R);
    for (int q = 0; q < 9; ++q) dinv[(int64_t)i * 9 + q] = R[q];
  }
}

// ---- line search: energy and CCD over the swept candidates --------------------------------
// sum over candidates of h^2 kappa b(d) at x + alpha d, and how many touch (d == 0)
__global__ void __launch_bounds__(kBlock) k_pair_energy(const int2* __restrict__ pt, int npt,
                                                        const int2* __restrict__ ee, int nee,
                                                        const int4* __restrict__ faces,
                                                        const int4* __restrict__ edges, const Vec4d* __restrict__ x,
                                                        const Vec4d* __restrict__ d, double alpha, double h2kappa,
                                                        double dhat, GridReduce gr, double* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[2] = {0.0, 0.0};
  if (idx < npt + nee) {
    const int kind = idx < npt ? 0 : 1;
    int v[4];
    pair_vertices(kind, kind == 0 ? pt[idx] : ee[idx - npt], faces, edges, v);
    D3 P[4];
    for (int a = 0; a < 4; ++a) P[a] = pos(x, d, alpha, v[a]);
    const double dist = cgeom::pair_distance(kind, P);
    if (!(dist >= 1e-300)) acc[1] = 1.0;
    else if (dist < dhat) acc[0] = h2kappa * bar_b(dist, dhat);
  }
  if (grid_sum<2>(acc, gr, RS_CONTACT) && threadIdx.x == 0) {
    out[0] = acc[0];
    out[1] = acc[1];
  }
}

// conservative advancement of one candidate over x -> x + d; the smallest
// fraction below 1 goes to *tmin (as the bit pattern of a non-negative double)
__global__ void k_pair_ccd(const int2* __restrict__ pt, int npt, const int2* __restrict__ ee, int nee,
                           const int4* __restrict__ faces, const int4* __restrict__ edges,
                           const Vec4d* __restrict__ x, const Vec4d* __restrict__ d, double* __restrict__ tmin) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npt + nee) return;
  const int kind = idx < npt ? 0 : 1;
  const int split = kind == 0 ? 1 : 2;  // vertices of the first primitive
  int v[4];
  pair_vertices(kind, kind == 0 ? pt[idx] : ee[idx - npt], faces, edges, v);
  D3 P0[4], dP[4];
  for (int a = 0; a < 4; ++a) {
    P0[a] = pos(x, nullptr, 0.0, v[a]);
    const Vec4d q = d[v[a]];
    dP[a] = D3{q.x, q.y, q.z};
  }
  // additive bound: displacements relative to the pair's mean displacement
  const D3 mean = cgeom::scl(0.25, cgeom::add(cgeom::add(dP[0], dP[1]), cgeom::add(dP[2], dP[3])));
  double m1 = 0.0, m2 = 0.0;
  for (int a = 0; a < 4; ++a) {
    const D3 r = cgeom::sub(dP[a], mean);
    const double l = sqrt(cgeom::dot(r, r));
    if (a < split) m1 = fmax(m1, l);
    else m2 = fmax(m2, l);
  }
  const double L = m1 + m2;
  if (!(L > 0.0)) return;  // a common translation keeps the distance
  const double d0 = cgeom::pair_distance(kind, P0);
  const double floor_d = kCcdS * d0;
  double t = 0.0, dist = d0;
  D3 P[4];
  for (int it = 0; it < kCcdMaxIter; ++it) {
    const double step = (dist - floor_d) / L;
    if (step <= kCcdRtol) break;
    if (t + step >= 1.0) {
      for (int a = 0; a < 4; ++a) P[a] = cgeom::add(P0[a], dP[a]);
      if (cgeom::pair_distance(kind, P) >= floor_d * (1.0 - 1e-12)) t = 1.0;
      break;
    }
    for (int a = 0; a < 4; ++a) P[a] = cgeom::add(P0[a], cgeom::scl(t + step, dP[a]));
    const double dn = cgeom::pair_distance(kind, P);
    if (dn < floor_d * (1.0 - 1e-12)) break;  // only rounding can cause this
    t += step;
    dist = dn;
  }
  if (t < 1.0) atomic_min_nonneg(tmin, t);
}

// ---- friction between bodies (Eq. IP term D), lagged at x^t ------------------------------
// The ground friction with the plane replaced by each pair's closest points:
// the pairs within dhat at x^t keep, for the whole step, the weights w of
// their closest-point difference, its unit normal n and mu lambda with
// lambda = -kappa b'(d); D = sum mu lambda f0(|u|), u = (I - n n^T)
// sum_j w_j (x_j - x_j^t).

// one thread per pair within dhat at x^t: its four vertices, w, n and mu lambda
__global__ void k_friction_lag(const int2* __restrict__ pt, int npt, const int2* __restrict__ ee, int nee,
                               const int4* __restrict__ faces, const int4* __restrict__ edges,
                               const Vec4d* __restrict__ xt, double mu, double kappa, double dhat,
                               int4* __restrict__ fv, double* __restrict__ fw) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npt + nee) return;
  const int kind = idx < npt ? 0 : 1;
  int v[4];
  pair_vertices(kind, kind == 0 ? pt[idx] : ee[idx - npt], faces, edges, v);
  D3 P[4];
  for (int a = 0; a < 4; ++a) P[a] = pos(xt, nullptr, 0.0, v[a]);
  double w[4];
  D3 n;
  const double d = cgeom::friction_frame(kind, P, w, n);
  fv[idx] = make_int4(v[0], v[1], v[2], v[3]);
  double* o = fw + 8 * (int64_t)idx;
  for (int j = 0; j < 4; ++j) o[j] = w[j];
  o[4] = n.x;
  o[5] = n.y;
  o[6] = n.z;
  o[7] = mu * fric_lambda(d, dhat, kappa);
}

// a lagged pair's slip at x (+ alpha d, d nullable)
__device__ __forceinline__ double friction_pair_slip(const int (&v)[4], const double* o, const Vec4d* __restrict__ x,
                                                     const Vec4d* __restrict__ d, double alpha,
                                                     const Vec4d* __restrict__ xt, D3& u) {
  const double w[4] = {o[0], o[1], o[2], o[3]};
  D3 dx[4];
  for (int j = 0; j < 4; ++j) dx[j] = cgeom::sub(pos(x, d, alpha, v[j]), pos(xt, nullptr, 0.0, v[j]));
  return cgeom::friction_slip(w, D3{o[4], o[5], o[6]}, dx, u);
}

// one thread per (lagged pair, vertex a, vertex b), as k_pair_scatter: the
// block w_a w_b mu lambda K at x into the coupling table and, for b = 0, the
// gradient mu lambda (f1(y)/y) w_a u of vertex a into cgrad (Dirichlet
// vertices left out)
__global__ void k_friction_scatter(const int4* __restrict__ fv, const double* __restrict__ fw, int nfr,
                                   const Vec4d* __restrict__ x, const Vec4d* __restrict__ xt,
                                   const uint8_t* __restrict__ pinned, double eps, Vec4d* __restrict__ cgrad,
                                   CouplingView C) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 16 * (int64_t)nfr) return;
  const int idx = (int)(t >> 4), a = (int)(t >> 2) & 3, b = (int)t & 3;
  const int4 v4 = fv[idx];
  const int v[4] = {v4.x, v4.y, v4.z, v4.w};
  if (pinned[v[a]] || pinned[v[b]]) return;
  const double* o = fw + 8 * (int64_t)idx;
  const double mul = o[7];
  if (!(mul > 0.0)) return;
  D3 u;
  const double y = friction_pair_slip(v, o, x, nullptr, 0.0, xt, u);
  const double ratio = fric_ratio(y, eps), slope = fric_slope(y, eps);
  if (b == 0 && o[a] != 0.0) {
    const double s = mul * ratio * o[a];
    atomicAdd(&cgrad[v[a]].x, s * u.x);
    atomicAdd(&cgrad[v[a]].y, s * u.y);
    atomicAdd(&cgrad[v[a]].z, s * u.z);
  }
  const double ww = mul * o[a] * o[b];
  if (ww == 0.0) return;
  double K[9];
  cgeom::friction_block(D3{o[4], o[5], o[6]}, u, y, ratio, slope, K);
  const int s = coupling_slot(C, v[a], v[b]);
  if (s < 0) return;
  for (int q = 0; q < 9; ++q) atomicAdd(C.val + 9 * (int64_t)s + q, ww * K[q]);
}

// sum over the lagged pairs of h^2 mu lambda f0(|u|) at x + alpha d
__global__ void __launch_bounds__(kBlock) k_friction_energy(const int4* __restrict__ fv, const double* __restrict__ fw,
                                                            int nfr, const Vec4d* __restrict__ x,
                                                            const Vec4d* __restrict__ d, double alpha,
                                                            const Vec4d* __restrict__ xt, double eps, double h2,
                                                            GridReduce gr, double* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  double acc[1] = {0.0};
  if (idx < nfr) {
    const double* o = fw + 8 * (int64_t)idx;
    if (o[7] > 0.0) {
      const int4 v4 = fv[idx];
      const int v[4] = {v4.x, v4.y, v4.z, v4.w};
      D3 u;
      const double y = friction_pair_slip(v, o, x, d, alpha, xt, u);
      acc[0] = h2 * o[7] * fric_f0(y, eps);
    }
  }
  if (grid_sum<1>(acc, gr, RS_CONTACT) && threadIdx.x == 0) out[0] = acc[0];
}

// ---- coarse operator: U_i^T H_ij U_j of the cross-body blocks ----------------------------
// one 144-thread block per cross-body coupling (i, j) with H_ij in slot s:
// for handles a of i and b of j, entry (12a + 4c + l, 12b + 4e + m) gains
// phi_a(i) abar_l(i) H_ij[c][e] phi_b(j) abar_m(j), abar = [1, X - o]
template <typename MT>
__global__ void __launch_bounds__(144) k_galerkin_contact(const int4* __restrict__ xc, int nxc,
                                                          const int* __restrict__ vrow, const int* __restrict__ vh,
                                                          const double* __restrict__ vphi,
                                                          const double* __restrict__ origins,
                                                          const Vec4d* __restrict__ X, const MT* __restrict__ val,
                                                          int r, double* __restrict__ Ac) {
  const int e = blockIdx.x;
  if (e >= nxc) return;
  const int4 c4 = xc[e];
  const int i = c4.x, j = c4.y;
  const int64_t slot = c4.z;
  const int t = threadIdx.x;
  const int c = t / 48, l = (t / 12) % 4, ce = (t % 12) / 4, m = t % 4;
  const double h = load_as<double>(val[(slot >> 5) * 288 + (3 * c + ce) * 32 + (slot & 31)]);
  const Vec4d Xi = X[i], Xj = X[j];
  for (int p = vrow[i]; p < vrow[i + 1]; ++p) {
    const int a = vh[p];
    const double pa = vphi[p];
    const double al = l == 0 ? pa : pa * (l == 1 ? Xi.x - origins[3 * a] : l == 2 ? Xi.y - origins[3 * a + 1]
                                                                                    : Xi.z - origins[3 * a + 2]);
    for (int q = vrow[j]; q < vrow[j + 1]; ++q) {
      const int b = vh[q];
      const double pb = vphi[q];
      const double bm = m == 0 ? pb : pb * (m == 1 ? Xj.x - origins[3 * b] : m == 2 ? Xj.y - origins[3 * b + 1]
                                                                                     : Xj.z - origins[3 * b + 2]);
      atomicAdd(Ac + (int64_t)(12 * a + 4 * c + l) * r + 12 * b + 4 * ce + m, al * h * bm);
    }
  }
}

// ---- per-pair derivatives for testing -------------------------------------------------------
// pairs given by their vertex positions X [P][4][3]: distance, grad d [12],
// Hess d [144] and the projected barrier Hessian [144], by the same warp
// code as the assembly
__global__ void __launch_bounds__(32 * kPairWarps) k_pair_derivatives(const int* __restrict__ kind,
                                                                      const double* __restrict__ X, int n,
                                                                      double kappa, double dhat,
                                                                      double* __restrict__ dist,
                                                                      double* __restrict__ gd,
                                                                      double* __restrict__ Hd,
                                                                      double* __restrict__ Hb) {
  __shared__ PairWarp sw[kPairWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * kPairWarps + warp;
  if (p >= n) return;
  PairWarp& W = sw[warp];
  D3 P[4];
  for (int a = 0; a < 4; ++a) P[a] = D3{X[12 * p + 3 * a], X[12 * p + 3 * a + 1], X[12 * p + 3 * a + 2]};
  pair_eval_warp(kind[p], P, kappa, dhat, W, lane, Hd + 144 * (int64_t)p, gd + 12 * (int64_t)p);
  if (lane == 0) dist[p] = cgeom::pair_distance(kind[p], P);
  for (int t = lane; t < 144; t += 32) Hb[144 * (int64_t)p + t] = W.A[t];
}

// ---- host side -------------------------------------------------------------------------------
static inline int nblocks(int64_t n, int b = kBlock) { return (int)std::max<int64_t>((n + b - 1) / b, 1); }

static int pow2_at_least(int64_t v) {
  int b = 0;
  while (((int64_t)1 << b) < v) ++b;
  return b;
}

void contact_free(mls_ctx* ctx) {
  ContactState& cs = ctx->cs;
  void* bufs[] = {cs.faces, cs.edges, cs.sverts, cs.row_len0, cs.head, cs.ent, cs.next, cs.boxes, cs.cnt,
                  cs.pt,    cs.ee,    cs.spt,    cs.see,      cs.ckey, cs.cval, cs.xc,  cs.cgrad, cs.ccd,
                  cs.pg,    cs.pH,    cs.bbox,   cs.fpt,      cs.fee,  cs.fv,   cs.fw};
  for (void* p : bufs) dfree(ctx, p);
  int* keep = cs.cnt_host;  // pinned, freed with the context
  cs = ContactState{};
  cs.cnt_host = keep;
}

void contact_invalidate(mls_ctx* ctx) { ctx->cs.sweep_valid = false; }

static mls_status regrow(mls_ctx* ctx, void** p, size_t bytes) {
  dfree(ctx, *p);
  *p = nullptr;
  return dalloc(ctx, p, bytes);
}

static mls_status read_counters(mls_ctx* ctx) {
  ContactState& cs = ctx->cs;
  mls_status st = cuda_check(ctx, cudaMemcpyAsync(cs.cnt_host, cs.cnt, sizeof(int) * kCntWords, cudaMemcpyDeviceToHost,
                                                  ctx->stream), "contact counters");
  if (st != MLS_OK) return st;
  return cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "contact sync");
}

// Broad phase over x (d null: pairs within dhat at x) or over the segment
// x -> x + d (every candidate), into (pt, ee); grows the grid and the pair
// buffers until everything fits.
static mls_status broad_phase(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, int2** pt, int2** ee, int64_t* cap,
                              int* npt, int* nee) {
  ContactState& cs = ctx->cs;
  double cell = std::max(cs.cell0, 2.0 * cs.dhat);
  mls_status st;
  for (int attempt = 0; attempt < 24; ++attempt) {
    if ((st = cuda_check(ctx, cudaMemsetAsync(cs.cnt, 0, sizeof(int) * kCntWords, ctx->stream), "counters")) != MLS_OK)
      return st;
    if ((st = cuda_check(ctx, cudaMemsetAsync(cs.head, 0xFF, sizeof(int) << (cs.hbits + 1), ctx->stream), "grid")) !=
        MLS_OK)
      return st;
    const bool pre = cs.nbody <= kMaxBodyBoxes;
    if (pre) {
      if ((st = cuda_check(ctx, cudaMemsetAsync(cs.bbox, 0xFF, sizeof(unsigned long long) * 3 * cs.nbody, ctx->stream),
                           "body boxes")) != MLS_OK)
        return st;
      if ((st = cuda_check(ctx, cudaMemsetAsync(cs.bbox + 3 * cs.nbody, 0, sizeof(unsigned long long) * 3 * cs.nbody,
                                                ctx->stream), "body boxes")) != MLS_OK)
        return st;
      ++ctx->launches;
      k_body_boxes<<<nblocks(cs.nsv), kBlock, 0, ctx->stream>>>(cs.sverts, cs.nsv, cs.nbody, x, d, cs.bbox,
                                                                 cs.bbox + 3 * cs.nbody);
    }
    GridView G{cs.nf, cs.ne, cs.nsv, cs.nbody, cs.faces, cs.edges, cs.sverts, cs.head, (1 << cs.hbits) - 1, cs.ent,
               cs.next, cs.ecap, cs.boxes, cs.cnt, pre ? cs.bbox : nullptr, pre ? cs.bbox + 3 * cs.nbody : nullptr,
               1.0 / cell, cs.dhat};
    ++ctx->launches;
    k_grid_insert<<<nblocks(cs.nf + cs.ne), kBlock, 0, ctx->stream>>>(G, x, d);
    ++ctx->launches;
    k_grid_query<<<nblocks(cs.nsv + cs.ne), kBlock, 0, ctx->stream>>>(G, x, d, PairOut{*pt, *ee, *cap});
    if ((st = cuda_check(ctx, cudaGetLastError(), "contact broad phase")) != MLS_OK) return st;
    if ((st = read_counters(ctx)) != MLS_OK) return st;
    const int* c = cs.cnt_host;
    if (c[kCntFlags] & kFlagRange) return fail(ctx, MLS_ENONFINITE, "contact broad phase: positions out of range");
    if (c[kCntFlags] & kFlagSpan) {  // boxes larger than the grid allows: coarser cells
      cell *= 2.0;
      continue;
    }
    if (c[kCntEnt] > cs.ecap) {
      cs.ecap = (int64_t)c[kCntEnt] * 3 / 2 + 1024;
      cs.hbits = pow2_at_least(2 * cs.ecap);
      if ((st = regrow(ctx, (void**)&cs.ent, sizeof(int4) * cs.ecap)) != MLS_OK) return st;
      if ((st = regrow(ctx, (void**)&cs.next, sizeof(int) * cs.ecap)) != MLS_OK) return st;
      if ((st = regrow(ctx, (void**)&cs.head, sizeof(int) << (cs.hbits + 1))) != MLS_OK) return st;
      continue;
    }
    if (c[kCntPT] > *cap || c[kCntEE] > *cap) {
      *cap = (int64_t)std::max(c[kCntPT], c[kCntEE]) * 3 / 2 + 1024;
      if ((st = regrow(ctx, (void**)pt, sizeof(int2) * *cap)) != MLS_OK) return st;
      if ((st = regrow(ctx, (void**)ee, sizeof(int2) * *cap)) != MLS_OK) return st;
      continue;
    }
    *npt = c[kCntPT];
    *nee = c[kCntEE];
    return MLS_OK;
  }
  return fail(ctx, MLS_ENOMEM, "contact broad phase did not settle");
}

static mls_status contact_sweep(mls_ctx* ctx, const Vec4d* x, const Vec4d* d) {
  ContactState& cs = ctx->cs;
  if (cs.sweep_valid && cs.sweep_x == x && cs.sweep_d == d) return MLS_OK;
  mls_status st = broad_phase(ctx, x, d, &cs.spt, &cs.see, &cs.scap, &cs.nspt, &cs.nsee);
  if (st != MLS_OK) return st;
  cs.sweep_valid = true;
  cs.sweep_x = x;
  cs.sweep_d = d;
  return MLS_OK;
}

mls_status contact_assemble(mls_ctx* ctx, const Vec4d* x) {
  ContactState& cs = ctx->cs;
  if (!cs.on) return MLS_OK;
  mls_status st = broad_phase(ctx, x, nullptr, &cs.pt, &cs.ee, &cs.pcap, &cs.npt, &cs.nee);
  if (st != MLS_OK) return st;
  const int np = cs.npt + cs.nee;
  // every pair (and every lagged friction pair) adds at most 16 vertex
  // couplings; the table stays at most half full
  const int64_t need = std::max<int64_t>(64, 32 * ((int64_t)np + cs.nfr));
  if (need > INT32_MAX / 2) return fail(ctx, MLS_ENOMEM, "too many contact pairs");
  if (cs.ccap < need) {
    cs.ccap = 1 << pow2_at_least(need);
    cs.xcap = cs.ccap;
    if ((st = regrow(ctx, (void**)&cs.ckey, sizeof(unsigned long long) * cs.ccap)) != MLS_OK) return st;
    if ((st = regrow(ctx, (void**)&cs.cval, sizeof(double) * 9 * cs.ccap)) != MLS_OK) return st;
    if ((st = regrow(ctx, (void**)&cs.xc, sizeof(int4) * cs.xcap)) != MLS_OK) return st;
  }
  if (np > cs.pbuf_cap) {
    cs.pbuf_cap = np + np / 2 + 256;
    if ((st = regrow(ctx, (void**)&cs.pg, sizeof(double) * 12 * cs.pbuf_cap)) != MLS_OK) return st;
    if ((st = regrow(ctx, (void**)&cs.pH, sizeof(double) * 144 * cs.pbuf_cap)) != MLS_OK) return st;
  }
  if ((st = cuda_check(ctx, cudaMemsetAsync(cs.ckey, 0xFF, sizeof(unsigned long long) * cs.ccap, ctx->stream),
                       "coupling keys")) != MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(cs.cval, 0, sizeof(double) * 9 * cs.ccap, ctx->stream),
                       "coupling values")) != MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(cs.cgrad, 0, sizeof(Vec4d) * ctx->n, ctx->stream),
                       "contact gradient")) != MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaMemsetAsync(cs.cnt, 0, sizeof(int) * kCntWords, ctx->stream), "counters")) != MLS_OK)
    return st;
  const CouplingView C{cs.ckey, cs.cval, cs.ccap - 1, cs.cnt + kCntFlags};
  if (np > 0) {
    ++ctx->launches;
    k_pair_eval<<<nblocks(np, kPairWarps), 32 * kPairWarps, 0, ctx->stream>>>(cs.pt, cs.npt, cs.ee, cs.nee, cs.faces,
                                                                              cs.edges, x, cs.kappa, cs.dhat, cs.pg,
                                                                              cs.pH);
    ++ctx->launches;
    k_pair_scatter<<<nblocks(16 * (int64_t)np), kBlock, 0, ctx->stream>>>(cs.pt, cs.npt, cs.ee, cs.nee, cs.faces,
                                                                          cs.edges, ctx->pinned, cs.pg, cs.pH,
                                                                          cs.cgrad, C);
  }
  if (cs.nfr > 0) {
    ++ctx->launches;
    k_friction_scatter<<<nblocks(16 * (int64_t)cs.nfr), kBlock, 0, ctx->stream>>>(
        cs.fv, cs.fw, cs.nfr, x, ctx->xt, ctx->pinned, ctx->fric_eps_v * ctx->h_step, cs.cgrad, C);
  }
  ++ctx->launches;
  k_contact_reset_rows<<<nblocks(cs.nsv), kBlock, 0, ctx->stream>>>(cs.sverts, cs.nsv, ctx->slice_ptr, cs.row_len0,
                                                                     ctx->row_len, ctx->col);
  cs.nxc = 0;
  return cuda_check(ctx, cudaGetLastError(), "contact pairs");
}

// The friction pairs of a step: the pairs within dhat at x^t, with their
// frames and normal forces (friction between bodies needs mu > 0 from
// mls_set_friction); called once per timestep before the Newton loop
mls_status contact_friction_lag(mls_ctx* ctx) {
  ContactState& cs = ctx->cs;
  cs.nfr = 0;
  if (!cs.on || !(ctx->fric_mu > 0.0)) return MLS_OK;
  int npt = 0, nee = 0;
  mls_status st = broad_phase(ctx, ctx->xt, nullptr, &cs.fpt, &cs.fee, &cs.fbcap, &npt, &nee);
  if (st != MLS_OK) return st;
  const int np = npt + nee;
  if (np > cs.fcap) {
    cs.fcap = np + np / 2 + 256;
    if ((st = regrow(ctx, (void**)&cs.fv, sizeof(int4) * cs.fcap)) != MLS_OK) return st;
    if ((st = regrow(ctx, (void**)&cs.fw, sizeof(double) * 8 * cs.fcap)) != MLS_OK) return st;
  }
  if (np > 0) {
    ++ctx->launches;
    k_friction_lag<<<nblocks(np), kBlock, 0, ctx->stream>>>(cs.fpt, npt, cs.fee, nee, cs.faces, cs.edges, ctx->xt,
                                                            ctx->fric_mu, cs.kappa, cs.dhat, cs.fv, cs.fw);
    if ((st = cuda_check(ctx, cudaGetLastError(), "k_friction_lag")) != MLS_OK) return st;
  }
  cs.nfr = np;
  return MLS_OK;
}

template <typename MT, typename VT>
static void launch_merge(mls_ctx* ctx, void* val, void* dinv, bool record) {
  ContactState& cs = ctx->cs;
  const CouplingView C{cs.ckey, cs.cval, cs.ccap - 1, cs.cnt + kCntFlags};
  ++ctx->launches;
  k_contact_merge<MT, VT><<<nblocks(cs.ccap), kBlock, 0, ctx->stream>>>(
      C, ctx->slice_ptr, cs.row_len0, ctx->row_len, ctx->col, (MT*)val, (VT*)dinv, ctx->h * ctx->h,
      record ? cs.xc : nullptr, cs.cnt + kCntXc, cs.xcap);
}

mls_status contact_merge(mls_ctx* ctx, void* val, void* dinv, bool record) {
  ContactState& cs = ctx->cs;
  if (!cs.on || cs.npt + cs.nee + cs.nfr == 0) return MLS_OK;
  mls_status st;
  if (record &&
      (st = cuda_check(ctx, cudaMemsetAsync(cs.cnt + kCntXc, 0, sizeof(int), ctx->stream), "xc count")) != MLS_OK)
    return st;
  switch (ctx->opt.precision) {
    case MLS_FP64: launch_merge<double, double>(ctx, val, dinv, record); break;
    case MLS_MIXED_FP32: launch_merge<float, float>(ctx, val, dinv, record); break;
    default: launch_merge<__nv_bfloat16, float>(ctx, val, dinv, record); break;
  }
  if ((st = cuda_check(ctx, cudaGetLastError(), "k_contact_merge")) != MLS_OK) return st;
  if ((st = read_counters(ctx)) != MLS_OK) return st;
  const int flags = cs.cnt_host[kCntFlags];
  if (flags & kFlagSlots)
    return fail(ctx, MLS_ENOMEM, "contact: a surface vertex touches more vertices of other bodies than its spare "
                                 "slots hold (raise spare in mls_set_bodies)");
  if (flags & kFlagTable) return fail(ctx, MLS_ENOMEM, "contact coupling table full");
  if (record) cs.nxc = std::min(cs.cnt_host[kCntXc], cs.xcap);
  return MLS_OK;
}

mls_status contact_galerkin(mls_ctx* ctx, const void* val) {
  ContactState& cs = ctx->cs;
  if (!cs.on || cs.nxc == 0) return MLS_OK;
  const Basis& B = ctx->basis;
  const int r = 12 * B.m;
  ++ctx->launches;
  switch (ctx->opt.precision) {
    case MLS_FP64:
      k_galerkin_contact<double><<<cs.nxc, 144, 0, ctx->stream>>>(cs.xc, cs.nxc, B.vrow, B.vh, B.vphi, B.origins,
                                                                  ctx->X, (const double*)val, r, ctx->Ac);
      break;
    case MLS_MIXED_FP32:
      k_galerkin_contact<float><<<cs.nxc, 144, 0, ctx->stream>>>(cs.xc, cs.nxc, B.vrow, B.vh, B.vphi, B.origins,
                                                                 ctx->X, (const float*)val, r, ctx->Ac);
      break;
    default:
      k_galerkin_contact<__nv_bfloat16><<<cs.nxc, 144, 0, ctx->stream>>>(
          cs.xc, cs.nxc, B.vrow, B.vh, B.vphi, B.origins, ctx->X, (const __nv_bfloat16*)val, r, ctx->Ac);
      break;
  }
  return cuda_check(ctx, cudaGetLastError(), "k_galerkin_contact");
}

// pair energy (with h^2) at x + alpha d over the candidates of x -> x + d,
// and whether a pair touches
mls_status contact_energy(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double alpha, double* E, int* infeasible) {
  ContactState& cs = ctx->cs;
  *E = 0.0;
  *infeasible = 0;
  if (!cs.on) return MLS_OK;
  mls_status st = contact_sweep(ctx, x, d);
  if (st != MLS_OK) return st;
  if (cs.nfr > 0) {  // friction between bodies over the lagged pairs
    if (nblocks(cs.nfr) > kMaxPartials) return fail(ctx, MLS_EINVAL, "too many friction pairs for one reduction grid");
    ++ctx->launches;
    k_friction_energy<<<nblocks(cs.nfr), kBlock, 0, ctx->stream>>>(cs.fv, cs.fw, cs.nfr, x, d, alpha, ctx->xt,
                                                                   ctx->fric_eps_v * ctx->h_step, ctx->h * ctx->h,
                                                                   ctx->red, ctx->dscal + 12);
    if ((st = cuda_check(ctx, cudaGetLastError(), "k_friction_energy")) != MLS_OK) return st;
    if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 12, ctx->dscal + 12, sizeof(double),
                                              cudaMemcpyDeviceToHost, ctx->stream), "friction energy")) != MLS_OK)
      return st;
    if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "friction energy sync")) != MLS_OK) return st;
    *E = ctx->dscal_host[12];
  }
  const int np = cs.nspt + cs.nsee;
  if (np == 0) return MLS_OK;
  if (nblocks(np) > kMaxPartials) return fail(ctx, MLS_EINVAL, "too many contact candidates for one reduction grid");
  ++ctx->launches;
  k_pair_energy<<<nblocks(np), kBlock, 0, ctx->stream>>>(cs.spt, cs.nspt, cs.see, cs.nsee, cs.faces, cs.edges, x, d,
                                                         alpha, ctx->h * ctx->h * cs.kappa, cs.dhat, ctx->red,
                                                         ctx->dscal + 8);
  if ((st = cuda_check(ctx, cudaGetLastError(), "k_pair_energy")) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 8, ctx->dscal + 8, 2 * sizeof(double),
                                            cudaMemcpyDeviceToHost, ctx->stream), "pair energy")) != MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "pair energy sync")) != MLS_OK) return st;
  *E += ctx->dscal_host[8];
  *infeasible = ctx->dscal_host[9] > 0.5 ? 1 : 0;
  return MLS_OK;
}

mls_status contact_ccd(mls_ctx* ctx, const Vec4d* x, const Vec4d* d, double* t) {
  ContactState& cs = ctx->cs;
  *t = 1.0;
  if (!cs.on) return MLS_OK;
  mls_status st = contact_sweep(ctx, x, d);
  if (st != MLS_OK) return st;
  const int np = cs.nspt + cs.nsee;
  if (np == 0) return MLS_OK;
  const double one = 1.0;
  if ((st = cuda_check(ctx, cudaMemcpyAsync(cs.ccd, &one, sizeof(double), cudaMemcpyHostToDevice, ctx->stream),
                       "ccd init")) != MLS_OK)
    return st;
  ++ctx->launches;
  k_pair_ccd<<<nblocks(np, 128), 128, 0, ctx->stream>>>(cs.spt, cs.nspt, cs.see, cs.nsee, cs.faces, cs.edges, x, d,
                                                        cs.ccd);
  if ((st = cuda_check(ctx, cudaGetLastError(), "k_pair_ccd")) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemcpyAsync(ctx->dscal_host + 10, cs.ccd, sizeof(double), cudaMemcpyDeviceToHost,
                                            ctx->stream), "ccd readback")) != MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaStreamSynchronize(ctx->stream), "ccd sync")) != MLS_OK) return st;
  *t = ctx->dscal_host[10];
  return MLS_OK;
}

}  // namespace mls

extern "C" {

mls_status mls_set_bodies(mls_ctx* ctx, const int32_t* body, double dhat, double kappa, int32_t spare) {
  using namespace mls;
  if (!ctx) return MLS_EINVAL;
  if (ctx->n < 1) return fail(ctx, MLS_EINVAL, "set_bodies: no mesh uploaded");
  if (ctx->has_basis || ctx->cub_scale)
    return fail(ctx, MLS_EINVAL, "set_bodies: call before mls_upload_basis and mls_upload_cubature");
  const int n = ctx->n, t = ctx->t;
  if (body) {
    if (!(dhat > 0) || !(kappa > 0)) return fail(ctx, MLS_EINVAL, "set_bodies: dhat and kappa must be positive");
    if (spare < 0) return fail(ctx, MLS_EINVAL, "set_bodies: negative spare slot count");
    for (int v = 0; v < n; ++v)
      if (body[v] < 0) return fail(ctx, MLS_EINVAL, "set_bodies: negative body label");
  }
  contact_free(ctx);
  // buffers laid out by H's pattern are rebuilt with it
  void** sized[] = {&ctx->hval, &ctx->hval_lag, &ctx->ehess_lag, &ctx->dinv_lag, &ctx->ws_hsave};
  for (void** p : sized) {
    dfree(ctx, *p);
    *p = nullptr;
  }
  ctx->assembled = false;
  ContactState& cs = ctx->cs;
  std::vector<std::array<int, 4>> faces;   // a, b, c, body
  std::vector<std::array<int, 3>> edges;   // a, b, body
  std::vector<std::array<int, 2>> sverts;  // v, body
  std::vector<int> extra;
  if (body) {
    // faces that belong to one tet only, in the tet's vertex order
    static const int fidx[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
    std::vector<std::array<int, 4>> keys((size_t)4 * t);  // sorted vertices, face id
    for (int e = 0; e < t; ++e)
      for (int f = 0; f < 4; ++f) {
        int a = ctx->h_tets[4 * e + fidx[f][0]], b = ctx->h_tets[4 * e + fidx[f][1]],
            c = ctx->h_tets[4 * e + fidx[f][2]];
        if (a > b) std::swap(a, b);
        if (b > c) std::swap(b, c);
        if (a > b) std::swap(a, b);
        keys[(size_t)4 * e + f] = {a, b, c, 4 * e + f};
      }
    std::sort(keys.begin(), keys.end());
    for (size_t k = 0; k < keys.size();) {
      size_t k2 = k + 1;
      while (k2 < keys.size() && keys[k2][0] == keys[k][0] && keys[k2][1] == keys[k][1] && keys[k2][2] == keys[k][2])
        ++k2;
      if (k2 == k + 1) {
        const int e = keys[k][3] / 4, f = keys[k][3] % 4;
        const int a = ctx->h_tets[4 * e + fidx[f][0]], b = ctx->h_tets[4 * e + fidx[f][1]],
                  c = ctx->h_tets[4 * e + fidx[f][2]];
        faces.push_back({a, b, c, body[a]});
      }
      k = k2;
    }
    std::vector<std::array<int, 2>> ev;
    std::vector<int> vs;
    for (const auto& f : faces)
      for (int k = 0; k < 3; ++k) {
        const int a = f[k], b = f[(k + 1) % 3];
        ev.push_back({std::min(a, b), std::max(a, b)});
        vs.push_back(f[k]);
      }
    std::sort(ev.begin(), ev.end());
    ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    double len = 0.0;
    for (const auto& e : ev) {
      edges.push_back({e[0], e[1], body[e[0]]});
      double s = 0.0;
      for (int c = 0; c < 3; ++c) {
        const double dd = ctx->h_X[3 * (size_t)e[0] + c] - ctx->h_X[3 * (size_t)e[1] + c];
        s += dd * dd;
      }
      len += std::sqrt(s);
    }
    for (int v : vs) sverts.push_back({v, body[v]});
    extra.assign(n, 0);
    const int sp = spare > 0 ? spare : 32;
    for (int v : vs) extra[v] = sp;
    cs.spare = sp;
    cs.cell0 = ev.empty() ? 0.0 : len / (double)ev.size();
    cs.dhat = dhat;
    cs.kappa = kappa;
    cs.h_body.assign(body, body + n);
  }
  mls_status st = build_pattern(ctx, body ? &extra : nullptr);
  if (st != MLS_OK) return st;
  const size_t hbytes = (size_t)storage_bytes(ctx) * 288 * ctx->n_groups;
  if ((st = dalloc(ctx, &ctx->hval, hbytes)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemset(ctx->hval, 0, hbytes), "H init")) != MLS_OK) return st;
  if (!body) return MLS_OK;
  cs.nf = (int)faces.size();
  cs.ne = (int)edges.size();
  cs.nsv = (int)sverts.size();
  std::vector<int4> hf(cs.nf), he(cs.ne);
  std::vector<int2> hs(cs.nsv);
  for (int k = 0; k < cs.nf; ++k) hf[k] = make_int4(faces[k][0], faces[k][1], faces[k][2], faces[k][3]);
  for (int k = 0; k < cs.ne; ++k) he[k] = make_int4(edges[k][0], edges[k][1], edges[k][2], 0);
  for (int k = 0; k < cs.nsv; ++k) hs[k] = make_int2(sverts[k][0], sverts[k][1]);
  auto up = [&](void** dst, const void* src, size_t bytes) -> mls_status {
    mls_status s2 = dalloc(ctx, dst, std::max<size_t>(bytes, 16));
    if (s2 != MLS_OK || bytes == 0) return s2;
    return cuda_check(ctx, cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice), "surface upload");
  };
  if ((st = up((void**)&cs.faces, hf.data(), sizeof(int4) * hf.size())) != MLS_OK) return st;
  if ((st = up((void**)&cs.edges, he.data(), sizeof(int4) * he.size())) != MLS_OK) return st;
  if ((st = up((void**)&cs.sverts, hs.data(), sizeof(int2) * hs.size())) != MLS_OK) return st;
  if ((st = up((void**)&cs.row_len0, ctx->h_row_len.data(), sizeof(int) * n)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&cs.cgrad, sizeof(Vec4d) * n)) != MLS_OK) return st;
  if ((st = cuda_check(ctx, cudaMemset(cs.cgrad, 0, sizeof(Vec4d) * n), "contact gradient")) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&cs.cnt, sizeof(int) * kCntWords)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&cs.ccd, sizeof(double))) != MLS_OK) return st;
  if (!cs.cnt_host) {
    if (cudaMallocHost((void**)&cs.cnt_host, sizeof(int) * kCntWords) != cudaSuccess) {
      cudaGetLastError();
      cs.cnt_host = nullptr;
      return fail(ctx, MLS_ENOMEM, "pinned contact counters");
    }
    ctx->host_allocs.push_back(cs.cnt_host);
  }
  cs.ecap = 8 * (int64_t)(cs.nf + cs.ne) + 1024;
  cs.hbits = pow2_at_least(2 * cs.ecap);
  if ((st = dalloc(ctx, (void**)&cs.ent, sizeof(int4) * cs.ecap)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&cs.next, sizeof(int) * cs.ecap)) != MLS_OK) return st;
  if ((st = dalloc(ctx, (void**)&cs.head, sizeof(int) << (cs.hbits + 1))) != MLS_OK) return st;
  cs.nbody = *std::max_element(body, body + n) + 1;
  if (cs.nbody <= kMaxBodyBoxes &&
      (st = dalloc(ctx, (void**)&cs.bbox, sizeof(unsigned long long) * 6 * cs.nbody)) != MLS_OK)
    return st;
  if ((st = dalloc(ctx, (void**)&cs.boxes, sizeof(double) * 6 * std::max(cs.nf + cs.ne, 1))) != MLS_OK) return st;
  cs.pcap = cs.scap = 2 * (int64_t)(cs.nsv + cs.ne) + 1024;
  void** pb[] = {(void**)&cs.pt, (void**)&cs.ee, (void**)&cs.spt, (void**)&cs.see};
  for (void** p : pb)
    if ((st = dalloc(ctx, p, sizeof(int2) * cs.pcap)) != MLS_OK) return st;
  cs.on = true;
  return MLS_OK;
}

mls_status mls_contact_pairs(mls_ctx* ctx, const double* x, const double* d, int64_t cap, int32_t* pt_out,
                             int64_t* npt, int32_t* ee_out, int64_t* nee) {
  using namespace mls;
  if (!ctx) return MLS_EINVAL;
  ContactState& cs = ctx->cs;
  if (!cs.on) return fail(ctx, MLS_EINVAL, "contact_pairs: no bodies set");
  if (!x || cap < 0 || !npt || !nee || (cap > 0 && (!pt_out || !ee_out)))
    return fail(ctx, MLS_EINVAL, "contact_pairs: null argument");
  mls_status st;
  if ((st = launch_pack(ctx, x, ctx->xk)) != MLS_OK) return st;
  if (d && (st = launch_pack(ctx, d, ctx->dir)) != MLS_OK) return st;
  int np = 0, ne2 = 0;
  if (d) {
    if ((st = contact_sweep(ctx, ctx->xk, ctx->dir)) != MLS_OK) return st;
    np = cs.nspt;
    ne2 = cs.nsee;
  } else {
    if ((st = broad_phase(ctx, ctx->xk, nullptr, &cs.pt, &cs.ee, &cs.pcap, &cs.npt, &cs.nee)) != MLS_OK) return st;
    np = cs.npt;
    ne2 = cs.nee;
  }
  *npt = np;
  *nee = ne2;
  const int2* dp = d ? cs.spt : cs.pt;
  const int2* de = d ? cs.see : cs.ee;
  std::vector<int2> hp(np), hee(ne2);
  std::vector<int4> hf(cs.nf), hE(cs.ne);
  if (np && (st = cuda_check(ctx, cudaMemcpy(hp.data(), dp, sizeof(int2) * np, cudaMemcpyDeviceToHost), "pairs")) !=
                MLS_OK)
    return st;
  if (ne2 && (st = cuda_check(ctx, cudaMemcpy(hee.data(), de, sizeof(int2) * ne2, cudaMemcpyDeviceToHost), "pairs")) !=
                 MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaMemcpy(hf.data(), cs.faces, sizeof(int4) * cs.nf, cudaMemcpyDeviceToHost), "faces")) !=
      MLS_OK)
    return st;
  if ((st = cuda_check(ctx, cudaMemcpy(hE.data(), cs.edges, sizeof(int4) * cs.ne, cudaMemcpyDeviceToHost), "edges")) !=
      MLS_OK)
    return st;
  for (int64_t k = 0; k < std::min<int64_t>(np, cap); ++k) {
    const int4 f = hf[hp[k].y];
    pt_out[4 * k] = hp[k].x; pt_out[4 * k + 1] = f.x; pt_out[4 * k + 2] = f.y; pt_out[4 * k + 3] = f.z;
  }
  for (int64_t k = 0; k < std::min<int64_t>(ne2, cap); ++k) {
    const int4 a = hE[hee[k].x], b = hE[hee[k].y];
    ee_out[4 * k] = a.x; ee_out[4 * k + 1] = a.y; ee_out[4 * k + 2] = b.x; ee_out[4 * k + 3] = b.y;
  }
  return MLS_OK;
}

mls_status mls_contact_pair_derivatives(const int32_t* kind, const double* X, int32_t n, double kappa, double dhat,
                                        double* dist, double* grad, double* hess_d, double* hess_b) {
  using namespace mls;
  if (n < 0 || (n > 0 && (!kind || !X || !dist || !grad || !hess_d || !hess_b)) || !(dhat > 0) || !(kappa > 0))
    return MLS_EINVAL;
  if (n == 0) return MLS_OK;
  k_pair_derivatives<<<nblocks(n, kPairWarps), 32 * kPairWarps>>>(kind, X, n, kappa, dhat, dist, grad, hess_d,
                                                                   hess_b);
  if (cudaGetLastError() != cudaSuccess) return MLS_ECUDA;
  return cudaDeviceSynchronize() == cudaSuccess ? MLS_OK : MLS_ECUDA;
}

}  // extern "C"
