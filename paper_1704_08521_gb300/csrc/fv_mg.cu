// Multigrid solve of the pressure-correction equation (Section 3, step 1 of
// the SIMPLE-like loop: D G phi = r with d phi / dn = 0 on the walls).
//
// The equation is solved in its symmetric form A phi = b with
//   (A phi)_P = sum over the faces f of P of  a_f (phi_P - phi_nb(f)),
//   a_f = (area of f) / (distance between the centres across f),
//   b = -V (r - c),  c = sum(V r) / sum(V),
// V the cell volumes: A = -V D G on the stretched grid, b the right-hand side
// made compatible with the Neumann null space the way the tensor-product
// solve makes it (its null mode is the constant), and the solution is
// returned with zero volume-weighted mean, so both solvers return the same
// phi.
//
// Outer iteration: flexible conjugate gradients in float64 (Polak-Ribiere
// beta, which tolerates the rounding of a float32 preconditioner), stopped at
// ||b - A phi||_2 <= rtol ||b||_2.  Preconditioner: one float32 V-cycle.
//
// Hierarchy: full coarsening of every axis with more than two cells (coarse
// cell I = fine cells 2I and 2I+1; an odd count leaves a last coarse cell of
// one fine cell), until no axis has more than four cells.  Coarse operators
// are rediscretised from the coarse cells' widths and centre distances (the
// same a_f formula).  Prolongation: tensor product of 1-D linear
// interpolation between coarse cell centres in the stretched coordinate,
// constant beyond the first and last centre (the Neumann walls).
// Restriction: its transpose, so the integrated residual is conserved.
// Smoother: zebra line Gauss-Seidel, alternating the line direction -- the
// cosine-stretched grids have cells with aspect ratios of tens, for which
// point smoothers fail and line smoothers do not.  Each half-sweep solves
// every line of one colour (lines coloured like a checkerboard of their two
// transverse indices, so neighbour lines differ in colour) exactly, in
// place: lines of up to kPartMaxLine cells are split over up to 8 warps (the
// partition method, k_line_part), longer ones take one thread each (the
// Thomas recurrence, k_line).  Pre-smoothing x, y, z (colours 0, 1) and
// post-smoothing in the exact reverse order, so the V-cycle is a symmetric
// preconditioner.  Coarsest
// level (at most 4 cells per axis): exact solve by the separable eigenbases
// of the coarse operator (A = sum over axes of K_d (x) W_others, K_d E_d =
// W_d E_d Lambda_d), null mode dropped.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fv_internal.cuh"
#include "fvns_host.h"

namespace fv {

namespace {

constexpr int kMgMaxLevels = 16;
constexpr int kCoarseMax = 4;       // coarsest level: at most this many cells per axis
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 592;     // 4 x 148: fixed, so the reductions are deterministic

// ------------------------------------------------------------ host tables --
struct Axis1D {
  int n = 0;
  std::vector<double> x;   // faces, n + 1
  std::vector<double> w;   // widths
  std::vector<double> xc;  // centres
  std::vector<double> t;   // n + 1: 1 / (centre distance) at interior faces, 0 at walls
};

Axis1D axis_from_faces(const std::vector<double>& x) {
  Axis1D a;
  a.n = (int)x.size() - 1;
  a.x = x;
  a.w.resize(a.n);
  a.xc.resize(a.n);
  a.t.assign(a.n + 1, 0.0);
  for (int m = 0; m < a.n; ++m) {
    a.w[m] = x[m + 1] - x[m];
    a.xc[m] = 0.5 * (x[m] + x[m + 1]);
  }
  for (int f = 1; f < a.n; ++f) a.t[f] = 1.0 / (a.xc[f] - a.xc[f - 1]);
  return a;
}

// coarse faces: every other fine face, and the last one
Axis1D coarsen(const Axis1D& f) {
  if (f.n <= 2) return f;
  const int nc = (f.n + 1) / 2;
  std::vector<double> X(nc + 1);
  for (int I = 0; I < nc; ++I) X[I] = f.x[2 * I];
  X[nc] = f.x[f.n];
  return axis_from_faces(X);
}

// prolongation from coarse c to fine f along one axis: fine cell m takes
// (1 - w1[m]) x_c[c0[m]] + w1[m] x_c[c0[m] + 1] (w1 = 0 where it is the
// nearest-centre constant); the identity if the axis was not coarsened
void prolongation(const Axis1D& f, const Axis1D& c, std::vector<int>& c0, std::vector<double>& w1) {
  c0.assign(f.n, 0);
  w1.assign(f.n, 0.0);
  if (c.n == f.n) {
    for (int m = 0; m < f.n; ++m) c0[m] = m;
    return;
  }
  for (int m = 0; m < f.n; ++m) {
    const double p = f.xc[m];
    if (p <= c.xc[0]) { c0[m] = 0; continue; }
    if (p >= c.xc[c.n - 1]) { c0[m] = c.n - 1; continue; }
    int I = 0;
    while (I + 1 < c.n && c.xc[I + 1] < p) ++I;
    c0[m] = I;
    w1[m] = (p - c.xc[I]) / (c.xc[I + 1] - c.xc[I]);
  }
}

// restriction = prolongation transposed: coarse index I gathers from at most
// four fine cells (fine index, weight), weight 0 in the unused slots
void restriction(const std::vector<int>& c0, const std::vector<double>& w1, int nc,
                 std::vector<int>& rf, std::vector<double>& rw) {
  rf.assign((size_t)nc * 4, 0);
  rw.assign((size_t)nc * 4, 0.0);
  std::vector<int> cnt(nc, 0);
  auto add = [&](int I, int m, double wt) {
    if (wt == 0.0) return;
    const int q = cnt[I]++;
    rf[(size_t)I * 4 + q] = m;
    rw[(size_t)I * 4 + q] = wt;
  };
  for (int m = 0; m < (int)c0.size(); ++m) {
    add(c0[m], m, 1.0 - w1[m]);
    if (w1[m] != 0.0) add(c0[m] + 1, m, w1[m]);
  }
}

int count_levels(const int n[3]) {
  int m[3] = {n[0], n[1], n[2]};
  int L = 1;
  while (std::max(m[0], std::max(m[1], m[2])) > kCoarseMax && L < kMgMaxLevels) {
    for (int d = 0; d < 3; ++d)
      if (m[d] > 2) m[d] = (m[d] + 1) / 2;
    ++L;
  }
  return L;
}

// ---------------------------------------------------------- device views --
struct LevDev {
  int n[3];
  int64_t ncell;
  const float* w[3];
  const float* t[3];
  // transfer between this level and the next coarser one
  const int* pc0[3];     // per index of this level
  const float* pw1[3];
  const int* rf[3];      // per index of the coarser level, 4 slots
  const float* rw[3];
};

struct Fine64 {
  int n[3];
  int64_t ncell;
  const double* w[3];
  const double* t[3];
};

struct CoarseDev {
  int n[3];
  const float* E[3];     // n x n row-major, W-orthonormal eigenvectors (columns)
  const float* lam[3];
};

__device__ __forceinline__ void cell_ijk(int64_t c, const int n[3], int& i, int& j, int& k) {
  i = (int)(c % n[0]);
  const int64_t r = c / n[0];
  j = (int)(r % n[1]);
  k = (int)(r / n[1]);
}

// A x at cell (i, j, k) and the diagonal of A there
template <typename T, typename Lv>
__device__ __forceinline__ T apply_at(const Lv& L, const T* __restrict__ x, int i, int j, int k,
                                      int64_t c, T* diag) {
  const int nx = L.n[0], ny = L.n[1], nz = L.n[2];
  const int64_t sy = nx, sz = (int64_t)nx * ny;
  const T wx = L.w[0][i], wy = L.w[1][j], wz = L.w[2][k];
  const T ax0 = wy * wz * L.t[0][i], ax1 = wy * wz * L.t[0][i + 1];
  const T ay0 = wx * wz * L.t[1][j], ay1 = wx * wz * L.t[1][j + 1];
  const T az0 = wx * wy * L.t[2][k], az1 = wx * wy * L.t[2][k + 1];
  const T xp = x[c];
  T s = (ax0 + ax1 + ay0 + ay1 + az0 + az1) * xp;
  if (i > 0) s -= ax0 * x[c - 1];
  if (i + 1 < nx) s -= ax1 * x[c + 1];
  if (j > 0) s -= ay0 * x[c - sy];
  if (j + 1 < ny) s -= ay1 * x[c + sy];
  if (k > 0) s -= az0 * x[c - sz];
  if (k + 1 < nz) s -= az1 * x[c + sz];
  if (diag) *diag = ax0 + ax1 + ay0 + ay1 + az0 + az1;
  return s;
}

// --------------------------------------------------------- V-cycle kernels --
// One half-sweep of zebra line Gauss-Seidel along axis D: every line along
// D of colour `color` (the parity of its two transverse indices' sum) is
// solved exactly for the current values of its neighbour lines, which all
// have the other colour and are not written by this launch:
//   x_line += omega * D_line^-1 (b - A x)_line,
// D_line the tridiagonal part of A along the line.  In place.  One thread per
// line; the Thomas recurrence keeps its c' and d' in cb / db (same indexing
// as the cells).  Transverse indices: a (the faster one: i for y- and
// z-lines, j for x-lines) and b (k for x- and y-lines, j for z-lines); the
// thread's line has a = 2 t_a + ((b + color) & 1).
template <int D>
__global__ void __launch_bounds__(128) k_line(LevDev L, float* __restrict__ x,
                                              const float* __restrict__ b, float* __restrict__ cb,
                                              float* __restrict__ db, float omega, int color) {
  const int nx = L.n[0], ny = L.n[1];
  const int nl = L.n[D];
  const int na = D == 0 ? ny : nx;
  const int nb = D == 2 ? ny : L.n[2];
  const int ha = (na + 1) >> 1;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ha * nb) return;
  const int tb = (int)(t / ha);
  const int ta = 2 * (int)(t - (int64_t)tb * ha) + ((tb + color) & 1);
  if (ta >= na) return;
  // first cell of the line and the stride along it
  int i0, j0, k0;
  int64_t stride;
  if (D == 0) {
    i0 = 0; j0 = ta; k0 = tb; stride = 1;
  } else if (D == 1) {
    i0 = ta; j0 = 0; k0 = tb; stride = nx;
  } else {
    i0 = ta; j0 = tb; k0 = 0; stride = (int64_t)nx * ny;
  }
  const int64_t c00 = ((int64_t)k0 * ny + j0) * nx + i0;
  const float* tD = L.t[D];
  // the two widths across the line
  const float wa = D == 0 ? L.w[1][j0] : L.w[0][i0];
  const float wb = D == 2 ? L.w[1][j0] : L.w[2][k0];
  const float cross = wa * wb;
  constexpr int U = 4;
  float cp = 0.f, dp = 0.f;
  for (int m0 = 0; m0 < nl; m0 += U) {
    float res[U], dg[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + u;
      if (m < nl) {
        const int i = D == 0 ? m : i0, j = D == 1 ? m : j0, k = D == 2 ? m : k0;
        const int64_t c = c00 + (int64_t)m * stride;
        float diag;
        const float ax = apply_at<float>(L, x, i, j, k, c, &diag);
        res[u] = b[c] - ax;
        dg[u] = diag;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m0 + u;
      if (m < nl) {
        const int64_t c = c00 + (int64_t)m * stride;
        const float lo = -cross * tD[m], up = -cross * tD[m + 1];
        const float inv = 1.f / (dg[u] - lo * cp);
        const float cc = up * inv;
        const float dd = (res[u] - lo * dp) * inv;
        cb[c] = cc;
        db[c] = dd;
        cp = cc;
        dp = dd;
      }
    }
  }
  float dn = 0.f;
  for (int m1 = nl - 1; m1 >= 0; m1 -= U) {
    float cc[U], dd[U], xi[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m1 - u;
      if (m >= 0) {
        const int64_t c = c00 + (int64_t)m * stride;
        cc[u] = cb[c];
        dd[u] = db[c];
        xi[u] = x[c];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int m = m1 - u;
      if (m >= 0) {
        const int64_t c = c00 + (int64_t)m * stride;
        const float del = dd[u] - cc[u] * dn;
        x[c] = xi[u] + omega * del;
        dn = del;
      }
    }
  }
}

// The same half-sweep with each line split over P warps (the partition
// method for tridiagonal systems): a block owns 32 lines of the colour (one
// per lane) and P segments of each (one per warp).  Segment p of a line has
// rows [s, e) and couples to the rows s - 1 and e of its neighbours only
// through its first row's lower and its last row's upper coefficient.
//  1. forward over the segment: residuals r_m (kept in shared memory), the
//     inverse pivots 1/den_m of the segment's own tridiagonal matrix T (kept),
//     and the last rows of y = T^-1 r, v = T^-1 e_first, w = T^-1 e_last;
//  2. the same elimination from the bottom: the first rows of y, v, w;
//  3. warp 0 solves, per line, the 2P boundary unknowns (first and last row
//     of each segment): a block-tridiagonal system with 2 x 2 blocks;
//  4. each segment solves T x = r - (coupling to the neighbours' boundary
//     values) with the kept pivots and adds omega x to the line.
// Shared memory: r and the pivots as [row][lane] (conflict-free), the
// boundary values [P][8][lane].
template <int D>
__global__ void __launch_bounds__(256) k_line_part(LevDev L, float* __restrict__ x,
                                                   const float* __restrict__ b, float omega,
                                                   int color, int P) {
  extern __shared__ float ps[];
  const int nx = L.n[0], ny = L.n[1];
  const int nl = L.n[D];
  const int na = D == 0 ? ny : nx;
  const int nb = D == 2 ? ny : L.n[2];
  const int ha = (na + 1) >> 1;
  const int lane = threadIdx.x & 31, p = threadIdx.x >> 5;
  float* R = ps;                    // [nl][32]
  float* Q = ps + nl * 32;          // [nl][32] inverse pivots
  float* S = Q + nl * 32;           // [P][8][32]
  const int64_t t = (int64_t)blockIdx.x * 32 + lane;
  bool valid = t < (int64_t)ha * nb;
  int ta = 0, tb = 0;
  if (valid) {
    tb = (int)(t / ha);
    ta = 2 * (int)(t - (int64_t)tb * ha) + ((tb + color) & 1);
    valid = ta < na;
  }
  int i0, j0, k0;
  int64_t stride;
  if (D == 0) {
    i0 = 0; j0 = ta; k0 = tb; stride = 1;
  } else if (D == 1) {
    i0 = ta; j0 = 0; k0 = tb; stride = nx;
  } else {
    i0 = ta; j0 = tb; k0 = 0; stride = (int64_t)nx * ny;
  }
  const int64_t c00 = ((int64_t)k0 * ny + j0) * nx + i0;
  const float* tD = L.t[D];
  const float wa = valid ? (D == 0 ? L.w[1][j0] : L.w[0][i0]) : 0.f;
  const float wb = valid ? (D == 2 ? L.w[1][j0] : L.w[2][k0]) : 0.f;
  const float cross = wa * wb;
  const int s0 = (int)(((int64_t)p * nl) / P), e0 = (int)(((int64_t)(p + 1) * nl) / P);
  // coefficient of row m: lower -cross t[m], upper -cross t[m + 1]; the
  // diagonal is A's (all six faces)
  auto diag_at = [&](int m) {       // the expression apply_at evaluates
    const int i = D == 0 ? m : i0, j = D == 1 ? m : j0, k = D == 2 ? m : k0;
    const float wx = L.w[0][i], wy = L.w[1][j], wz = L.w[2][k];
    const float ax0 = wy * wz * L.t[0][i], ax1 = wy * wz * L.t[0][i + 1];
    const float ay0 = wx * wz * L.t[1][j], ay1 = wx * wz * L.t[1][j + 1];
    const float az0 = wx * wy * L.t[2][k], az1 = wx * wy * L.t[2][k + 1];
    return ax0 + ax1 + ay0 + ay1 + az0 + az1;
  };
  float yl = 0.f, vl = 0.f, wl = 0.f, yf = 0.f, vf = 0.f, wf = 0.f;
  const float lext = -cross * tD[s0], uext = -cross * tD[e0];
  if (valid) {
    // 1. forward
    float dy = 0.f, dv = 0.f, dw = 0.f, cprev = 0.f;
    constexpr int U = 4;
    for (int m0 = s0; m0 < e0; m0 += U) {
      float res[U], dg[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = m0 + u;
        if (m < e0) {
          const int i = D == 0 ? m : i0, j = D == 1 ? m : j0, k = D == 2 ? m : k0;
          const int64_t c = c00 + (int64_t)m * stride;
          float dgv;
          const float ax = apply_at<float>(L, x, i, j, k, c, &dgv);
          res[u] = b[c] - ax;
          dg[u] = dgv;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int m = m0 + u;
        if (m < e0) {
          const float lo = m > s0 ? -cross * tD[m] : 0.f;
          const float up = m < e0 - 1 ? -cross * tD[m + 1] : 0.f;
          const float inv = 1.f / (dg[u] - lo * cprev);
          dy = (res[u] - lo * dy) * inv;
          dv = ((m == s0 ? 1.f : 0.f) - lo * dv) * inv;
          dw = ((m == e0 - 1 ? 1.f : 0.f) - lo * dw) * inv;
          cprev = up * inv;
          R[m * 32 + lane] = res[u];
          Q[m * 32 + lane] = inv;
        }
      }
    }
    yl = dy; vl = dv; wl = dw;
    // 2. the same elimination from the bottom row up
    float ry = 0.f, rv = 0.f, rw = 0.f, gprev = 0.f;
    for (int m = e0 - 1; m >= s0; --m) {
      const float lo = m > s0 ? -cross * tD[m] : 0.f;
      const float up = m < e0 - 1 ? -cross * tD[m + 1] : 0.f;
      const float inv = 1.f / (diag_at(m) - up * gprev);
      const float r = R[m * 32 + lane];
      ry = (r - up * ry) * inv;
      rv = ((m == s0 ? 1.f : 0.f) - up * rv) * inv;
      rw = ((m == e0 - 1 ? 1.f : 0.f) - up * rw) * inv;
      gprev = lo * inv;
    }
    yf = ry; vf = rv; wf = rw;
  }
  float* Sp = S + (p * 8) * 32 + lane;
  Sp[0 * 32] = yf; Sp[1 * 32] = yl; Sp[2 * 32] = vf; Sp[3 * 32] = vl;
  Sp[4 * 32] = wf; Sp[5 * 32] = wl; Sp[6 * 32] = lext; Sp[7 * 32] = uext;
  __syncthreads();
  // 3. boundary unknowns X_q = (a_q, b_q) (first, last row of segment q):
  //    A_q X_{q-1} + X_q + C_q X_{q+1} = Y_q, A_q = lext_q [0 v_f; 0 v_l],
  //    C_q = uext_q [w_f 0; w_l 0]; block elimination, then back-substitution
  if (p == 0 && valid) {
    float Ch[8][4], Yh[8][2];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (q < P) {
        const float* Sq = S + (q * 8) * 32 + lane;
        const float qyf = Sq[0], qyl = Sq[32], qvf = Sq[64], qvl = Sq[96];
        const float qwf = Sq[128], qwl = Sq[160], ql = Sq[192], qu = Sq[224];
        // B = I - A_q Ch_{q-1}; A_q has only a second column (lext v_f, lext v_l)
        float b00 = 1.f, b01 = 0.f, b10 = 0.f, b11 = 1.f, y0 = qyf, y1 = qyl;
        if (q > 0) {
          const float a0 = ql * qvf, a1 = ql * qvl;        // A_q = [0 a0; 0 a1]
          // A_q Ch = [a0 Ch[1][:]; a1 Ch[1][:]] (row 1 of Ch: entries 2, 3)
          b00 -= a0 * Ch[q - 1][2]; b01 -= a0 * Ch[q - 1][3];
          b10 -= a1 * Ch[q - 1][2]; b11 -= a1 * Ch[q - 1][3];
          y0 -= a0 * Yh[q - 1][1];
          y1 -= a1 * Yh[q - 1][1];
        }
        const float det = b00 * b11 - b01 * b10;
        const float i00 = b11 / det, i01 = -b01 / det, i10 = -b10 / det, i11 = b00 / det;
        // C_q = [c0 0; c1 0] with c0 = uext w_f, c1 = uext w_l
        const float c0 = qu * qwf, c1 = qu * qwl;
        Ch[q][0] = i00 * c0 + i01 * c1; Ch[q][1] = 0.f;
        Ch[q][2] = i10 * c0 + i11 * c1; Ch[q][3] = 0.f;
        Yh[q][0] = i00 * y0 + i01 * y1;
        Yh[q][1] = i10 * y0 + i11 * y1;
      }
    }
    float xa = 0.f;                  // a_{q+1}
#pragma unroll
    for (int q = 7; q >= 0; --q) {
      if (q < P) {
        const float a = Yh[q][0] - Ch[q][0] * xa;
        const float bq = Yh[q][1] - Ch[q][2] * xa;
        S[(q * 8 + 0) * 32 + lane] = a;     // first row of segment q
        S[(q * 8 + 1) * 32 + lane] = bq;    // last row of segment q
        xa = a;
      }
    }
  }
  __syncthreads();
  if (!valid) return;
  // 4. the segment's rows from its modified right-hand side
  const float xprev = p > 0 ? S[((p - 1) * 8 + 1) * 32 + lane] : 0.f;
  const float xnext = p < P - 1 ? S[((p + 1) * 8 + 0) * 32 + lane] : 0.f;
  float d = 0.f;
  for (int m = s0; m < e0; ++m) {
    const float lo = m > s0 ? -cross * tD[m] : 0.f;
    float rhs = R[m * 32 + lane];
    if (m == s0) rhs -= lext * xprev;
    if (m == e0 - 1) rhs -= uext * xnext;
    d = (rhs - lo * d) * Q[m * 32 + lane];
    R[m * 32 + lane] = d;
  }
  float dn = 0.f;
  for (int m = e0 - 1; m >= s0; --m) {
    const float up = m < e0 - 1 ? -cross * tD[m + 1] : 0.f;
    const float del = R[m * 32 + lane] - up * Q[m * 32 + lane] * dn;
    const int64_t c = c00 + (int64_t)m * stride;
    x[c] += omega * del;
    dn = del;
  }
}

__global__ void k_resid32(LevDev L, const float* __restrict__ x, const float* __restrict__ b,
                          float* __restrict__ res) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(c, L.n, i, j, k);
    res[c] = b[c] - apply_at<float>(L, x, i, j, k, c, nullptr);
  }
}

// bc = R res (R = P^T), per coarse cell
__global__ void k_restrict(LevDev L, int nc0, int nc1, int nc2, const float* __restrict__ res,
                           float* __restrict__ bc) {
  const int64_t ncc = (int64_t)nc0 * nc1 * nc2;
  const int nx = L.n[0], ny = L.n[1];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int I = (int)(c % nc0);
    const int J = (int)((c / nc0) % nc1);
    const int K = (int)(c / ((int64_t)nc0 * nc1));
    float s = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const float wz = L.rw[2][K * 4 + r];
      if (wz == 0.f) continue;
      const int k = L.rf[2][K * 4 + r];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float wy = L.rw[1][J * 4 + q];
        if (wy == 0.f) continue;
        const int j = L.rf[1][J * 4 + q];
        const float* row = res + ((int64_t)k * ny + j) * nx;
        float sx = 0.f;
#pragma unroll
        for (int p = 0; p < 4; ++p) sx += L.rw[0][I * 4 + p] * row[L.rf[0][I * 4 + p]];
        s += wz * wy * sx;
      }
    }
    bc[c] = s;
  }
}

// x += P xc, per fine cell
__global__ void k_prolong_add(LevDev L, int nc0, int nc1, const float* __restrict__ xc,
                              float* __restrict__ x) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < L.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(c, L.n, i, j, k);
    const int I = L.pc0[0][i], J = L.pc0[1][j], K = L.pc0[2][k];
    const float a = L.pw1[0][i], bq = L.pw1[1][j], g = L.pw1[2][k];
    const int I1 = a != 0.f ? I + 1 : I, J1 = bq != 0.f ? J + 1 : J, K1 = g != 0.f ? K + 1 : K;
    auto at = [&](int kk, int jj, int ii) { return xc[((int64_t)kk * nc1 + jj) * nc0 + ii]; };
    const float v00 = (1.f - a) * at(K, J, I) + a * at(K, J, I1);
    const float v01 = (1.f - a) * at(K, J1, I) + a * at(K, J1, I1);
    const float v10 = (1.f - a) * at(K1, J, I) + a * at(K1, J, I1);
    const float v11 = (1.f - a) * at(K1, J1, I) + a * at(K1, J1, I1);
    x[c] += (1.f - g) * ((1.f - bq) * v00 + bq * v01) + g * ((1.f - bq) * v10 + bq * v11);
  }
}

// exact coarsest solve x = E Lambda^+ E^T b (3-D Kronecker), one block
__global__ void k_coarse(CoarseDev C, const float* __restrict__ b, float* __restrict__ x) {
  __shared__ float bh[kCoarseMax * kCoarseMax * kCoarseMax];
  const int nx = C.n[0], ny = C.n[1], nz = C.n[2];
  const int nc = nx * ny * nz;
  const int t = threadIdx.x;
  if (t < nc) {              // bh[c,b,a] = sum E_x[i][a] E_y[j][b] E_z[k][c] b[k][j][i] / lam
    const int a = t % nx, bb = (t / nx) % ny, cc = t / (nx * ny);
    float s = 0.f;
    for (int k = 0; k < nz; ++k)
      for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i)
          s += C.E[0][i * nx + a] * C.E[1][j * ny + bb] * C.E[2][k * nz + cc] *
               b[(k * ny + j) * nx + i];
    const float lam = C.lam[0][a] + C.lam[1][bb] + C.lam[2][cc];
    bh[t] = lam > 0.f ? s / lam : 0.f;
  }
  __syncthreads();
  if (t < nc) {
    const int i = t % nx, j = (t / nx) % ny, k = t / (nx * ny);
    float s = 0.f;
    for (int cc = 0; cc < nz; ++cc)
      for (int bb = 0; bb < ny; ++bb)
        for (int a = 0; a < nx; ++a)
          s += C.E[0][i * nx + a] * C.E[1][j * ny + bb] * C.E[2][k * nz + cc] *
               bh[(cc * ny + bb) * nx + a];
    x[t] = s;
  }
}

__global__ void k_round_cells(int64_t n, const double* __restrict__ in, float* __restrict__ out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    out[c] = (float)in[c];
}

__global__ void k_widen_cells(int64_t n, const float* __restrict__ in, double* __restrict__ out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    out[c] = (double)in[c];
}

// ---------------------------------------------------------- float64 CG part --
// scalar slots of the CG recurrences (device)
enum { S_RHO = 0, S_PQ, S_ALPHA, S_RR, S_RZ, S_RZO, S_BETA, S_VR, S_BB, S_VPHI, S_N };

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  return s;   // valid in thread 0
}

__device__ __forceinline__ double vol(const Fine64& F, int64_t c) {
  int i, j, k;
  cell_ijk(c, F.n, i, j, k);
  return F.w[0][i] * F.w[1][j] * F.w[2][k];
}

// part[block] = sum V r
__global__ void k_sum_vr(Fine64 F, const double* __restrict__ r, double* __restrict__ part) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < F.ncell;
       c += (int64_t)gridDim.x * blockDim.x)
    s += vol(F, c) * r[c];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// b = -V (r - c), c = S_VR / vtot; rcg = b (phi = 0) or b - A phi (guess);
// part[block] = sum b^2
__global__ void k_rhs(Fine64 F, const double* __restrict__ r, const double* __restrict__ s,
                      double vtot, const double* __restrict__ phi, double* __restrict__ rcg,
                      double* __restrict__ part) {
  __shared__ double sh[32];
  const double cm = s[S_VR] / vtot;
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < F.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double b = -vol(F, c) * (r[c] - cm);
    acc += b * b;
    double v = b;
    if (phi) {
      int i, j, k;
      cell_ijk(c, F.n, i, j, k);
      v -= apply_at<double>(F, phi, i, j, k, c, nullptr);
    }
    rcg[c] = v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// part2[block] = (sum r z, sum r zo)
__global__ void k_dots2(int64_t n, const double* __restrict__ r, const double* __restrict__ z,
                        const double* __restrict__ zo, double* __restrict__ part) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    const double rc = r[c];
    a += rc * z[c];
    b += rc * zo[c];
  }
  a = block_sum(a, sh);
  b = block_sum(b, sh);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = b;
  }
}

// q = A p, part[block] = sum p q
__global__ void k_apply64(Fine64 F, const double* __restrict__ p, double* __restrict__ q,
                          double* __restrict__ part) {
  __shared__ double sh[32];
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < F.ncell;
       c += (int64_t)gridDim.x * blockDim.x) {
    int i, j, k;
    cell_ijk(c, F.n, i, j, k);
    const double v = apply_at<double>(F, p, i, j, k, c, nullptr);
    q[c] = v;
    acc += p[c] * v;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// phi += alpha p, r -= alpha q, part[block] = sum r^2
__global__ void k_cg_step(int64_t n, const double* __restrict__ s, const double* __restrict__ p,
                          const double* __restrict__ q, double* __restrict__ phi,
                          double* __restrict__ r, double* __restrict__ part) {
  __shared__ double sh[32];
  const double al = s[S_ALPHA];
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x) {
    phi[c] += al * p[c];
    const double rv = r[c] - al * q[c];
    r[c] = rv;
    acc += rv * rv;
  }
  acc = block_sum(acc, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = acc;
}

// p = z + beta p
__global__ void k_cg_dir(int64_t n, const double* __restrict__ s, const double* __restrict__ z,
                         double* __restrict__ p) {
  const double be = s[S_BETA];
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    p[c] = z[c] + be * p[c];
}

// phi -= S_VPHI / vtot
__global__ void k_sub_mean(int64_t n, const double* __restrict__ s, double vtot,
                           double* __restrict__ phi) {
  const double m = s[S_VPHI] / vtot;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n;
       c += (int64_t)gridDim.x * blockDim.x)
    phi[c] -= m;
}

// one block: reduce the partials in a fixed order and run the scalar step
//   op 0: s[dst] = sum
//   op 1: (r z, r zo) pairs; beta = first ? 0 : (rz - rzo) / rho; rho = rz
//   op 2: s[S_PQ] = sum; alpha = rho / pq (0 if pq <= 0)
enum { OP_STORE = 0, OP_BETA = 1, OP_ALPHA = 2 };
__global__ void k_finalize(const double* __restrict__ part, int nblk, int op, int dst, int first,
                           double* __restrict__ s) {
  __shared__ double sh[32];
  double a = 0.0, b = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) {
    if (op == OP_BETA) {
      a += part[2 * q];
      b += part[2 * q + 1];
    } else {
      a += part[q];
    }
  }
  a = block_sum(a, sh);
  if (op == OP_BETA) b = block_sum(b, sh);
  if (threadIdx.x != 0) return;
  if (op == OP_STORE) {
    s[dst] = a;
  } else if (op == OP_BETA) {
    s[S_RZ] = a;
    s[S_RZO] = b;
    s[S_BETA] = first || s[S_RHO] == 0.0 ? 0.0 : (a - b) / s[S_RHO];
    s[S_RHO] = a;
  } else {
    s[S_PQ] = a;
    s[S_ALPHA] = a > 0.0 ? s[S_RHO] / a : 0.0;
  }
}

// ------------------------------------------------------------- the state --
struct MgLevelHost {
  Axis1D ax[3];
  LevDev dev;
  float* x[2] = {nullptr, nullptr};
  float* b = nullptr;
  float* res = nullptr;
  float* cb = nullptr;
  float* db = nullptr;
  int cur = 0;      // which x holds the level's iterate
};

}  // namespace

struct MgState {
  int nlev = 0;
  MgLevelHost lev[kMgMaxLevels];
  Fine64 fine;
  CoarseDev coarse;
  double vtot = 0.0;
  void* d_tab = nullptr;      // 1-D tables of all levels (floats, ints, doubles)
  void* d_work = nullptr;     // level arrays
  double* r = nullptr;        // CG vectors (float64, n_cell each)
  double* z[2] = {nullptr, nullptr};
  double* p = nullptr;
  double* q = nullptr;
  double* part = nullptr;     // 2 x kRedBlocks
  double* s = nullptr;        // S_N scalars
  double* h_s = nullptr;      // pinned mirror
};

namespace {

int blocks_for(int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 4 * 152 * 4));
}

fv_status build_mg(fv_grid* g) {
  MgState* M = new MgState();
  g->mg = M;
  const int n0[3] = {g->n[0], g->n[1], g->n[2]};
  M->nlev = count_levels(n0);
  for (int d = 0; d < 3; ++d) M->lev[0].ax[d] = axis_from_faces(g->h_x[d]);
  for (int l = 1; l < M->nlev; ++l)
    for (int d = 0; d < 3; ++d) M->lev[l].ax[d] = coarsen(M->lev[l - 1].ax[d]);
  // table layout: per level and axis w (n), t (n + 1), pw1 (n), rw (4 n_coarse) as
  // floats; pc0 (n), rf (4 n_coarse) as ints; level-0 w, t as doubles; the coarse
  // eigenbases and eigenvalues as floats
  std::vector<float> tf;
  std::vector<int> ti;
  std::vector<double> td;
  struct Off { size_t w, t, pw1, rw, pc0, rf; } off[kMgMaxLevels][3];
  for (int l = 0; l < M->nlev; ++l) {
    for (int d = 0; d < 3; ++d) {
      const Axis1D& a = M->lev[l].ax[d];
      Off& o = off[l][d];
      o.w = tf.size();
      for (double v : a.w) tf.push_back((float)v);
      o.t = tf.size();
      for (double v : a.t) tf.push_back((float)v);
      if (l + 1 < M->nlev) {
        std::vector<int> c0, rf;
        std::vector<double> w1, rw;
        const Axis1D& c = M->lev[l + 1].ax[d];
        prolongation(a, c, c0, w1);
        restriction(c0, w1, c.n, rf, rw);
        o.pw1 = tf.size();
        for (double v : w1) tf.push_back((float)v);
        o.rw = tf.size();
        for (double v : rw) tf.push_back((float)v);
        o.pc0 = ti.size();
        ti.insert(ti.end(), c0.begin(), c0.end());
        o.rf = ti.size();
        ti.insert(ti.end(), rf.begin(), rf.end());
      } else {
        o.pw1 = o.rw = o.pc0 = o.rf = 0;
      }
    }
  }
  size_t w64[3], t64[3];
  for (int d = 0; d < 3; ++d) {
    w64[d] = td.size();
    td.insert(td.end(), M->lev[0].ax[d].w.begin(), M->lev[0].ax[d].w.end());
    t64[d] = td.size();
    td.insert(td.end(), M->lev[0].ax[d].t.begin(), M->lev[0].ax[d].t.end());
  }
  // coarsest level: W-orthonormal eigenvectors of K_d E = W_d E Lambda
  size_t cE[3], cL[3];
  const int lc = M->nlev - 1;
  for (int d = 0; d < 3; ++d) {
    const Axis1D& a = M->lev[lc].ax[d];
    const int n = a.n;
    std::vector<double> dg(n, 0.0), e(n > 1 ? n - 1 : 1, 0.0), lam, Z;
    for (int f = 1; f < n; ++f) {
      dg[f - 1] += a.t[f];
      dg[f] += a.t[f];
      e[f - 1] = -a.t[f] / std::sqrt(a.w[f - 1] * a.w[f]);
    }
    for (int m = 0; m < n; ++m) dg[m] /= a.w[m];
    if (!sym_tridiag_eig(n, dg, e, lam, Z)) {
      set_error("multigrid: coarse eigensolve did not converge");
      return FV_ENOCONV;
    }
    // the null eigenvalue is zero in exact arithmetic: make it so
    int null = 0;
    for (int q = 1; q < n; ++q)
      if (std::fabs(lam[q]) < std::fabs(lam[null])) null = q;
    lam[null] = 0.0;
    cE[d] = tf.size();
    for (int m = 0; m < n; ++m)
      for (int q = 0; q < n; ++q) tf.push_back((float)(Z[(size_t)m * n + q] / std::sqrt(a.w[m])));
    cL[d] = tf.size();
    for (double v : lam) tf.push_back((float)std::max(v, 0.0));
  }
  const size_t bf = tf.size() * 4, bi = ti.size() * 4, bd = td.size() * 8;
  const size_t oi = (bf + 255) / 256 * 256, od = oi + (bi + 255) / 256 * 256;
  FV_CUDA(cudaMalloc(&M->d_tab, od + bd));
  char* base = (char*)M->d_tab;
  FV_CUDA(cudaMemcpy(base, tf.data(), bf, cudaMemcpyHostToDevice));
  if (bi) FV_CUDA(cudaMemcpy(base + oi, ti.data(), bi, cudaMemcpyHostToDevice));
  FV_CUDA(cudaMemcpy(base + od, td.data(), bd, cudaMemcpyHostToDevice));
  const float* F = (const float*)base;
  const int* I = (const int*)(base + oi);
  const double* Dd = (const double*)(base + od);
  // level arrays: x0, x1, b, res, cb, db per level
  size_t cells = 0;
  for (int l = 0; l < M->nlev; ++l) {
    int64_t nc = 1;
    for (int d = 0; d < 3; ++d) nc *= M->lev[l].ax[d].n;
    cells += (size_t)(nc + 63) / 64 * 64;
  }
  FV_CUDA(cudaMalloc(&M->d_work, cells * 6 * sizeof(float)));
  float* wp = (float*)M->d_work;
  for (int l = 0; l < M->nlev; ++l) {
    MgLevelHost& H = M->lev[l];
    LevDev& v = H.dev;
    int64_t nc = 1;
    for (int d = 0; d < 3; ++d) {
      v.n[d] = H.ax[d].n;
      nc *= v.n[d];
      v.w[d] = F + off[l][d].w;
      v.t[d] = F + off[l][d].t;
      const bool has = l + 1 < M->nlev;
      v.pw1[d] = has ? F + off[l][d].pw1 : nullptr;
      v.rw[d] = has ? F + off[l][d].rw : nullptr;
      v.pc0[d] = has ? I + off[l][d].pc0 : nullptr;
      v.rf[d] = has ? I + off[l][d].rf : nullptr;
    }
    v.ncell = nc;
    const size_t stride = (size_t)(nc + 63) / 64 * 64;
    H.x[0] = wp; wp += stride;
    H.x[1] = wp; wp += stride;
    H.b = wp; wp += stride;
    H.res = wp; wp += stride;
    H.cb = wp; wp += stride;
    H.db = wp; wp += stride;
  }
  for (int d = 0; d < 3; ++d) {
    M->fine.n[d] = g->n[d];
    M->fine.w[d] = Dd + w64[d];
    M->fine.t[d] = Dd + t64[d];
    M->coarse.n[d] = M->lev[lc].ax[d].n;
    M->coarse.E[d] = F + cE[d];
    M->coarse.lam[d] = F + cL[d];
  }
  M->fine.ncell = g->ncell;
  M->vtot = 1.0;
  for (int d = 0; d < 3; ++d) M->vtot *= g->h_x[d].back() - g->h_x[d].front();
  const size_t nb = (size_t)g->ncell * sizeof(double);
  double* cg = nullptr;
  FV_CUDA(cudaMalloc((void**)&cg, 5 * nb + (2 * kRedBlocks + S_N) * sizeof(double)));
  M->r = cg;
  M->z[0] = cg + g->ncell;
  M->z[1] = cg + 2 * g->ncell;
  M->p = cg + 3 * g->ncell;
  M->q = cg + 4 * g->ncell;
  M->part = cg + 5 * g->ncell;
  M->s = M->part + 2 * kRedBlocks;
  FV_CUDA(cudaMallocHost((void**)&M->h_s, S_N * sizeof(double)));
  FV_CUDA(cudaDeviceSynchronize());
  return FV_OK;
}

// lines of at most this many cells take the partitioned kernel (its shared
// memory grows with the line)
constexpr int kPartMaxLine = 640;

size_t part_smem(int nl, int P) { return sizeof(float) * ((size_t)2 * nl * 32 + (size_t)P * 8 * 32); }

fv_status set_part_attributes() {
  static bool done = false;
  if (!done) {
    const int bytes = (int)part_smem(kPartMaxLine, 8);
    FV_CUDA(cudaFuncSetAttribute(k_line_part<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    FV_CUDA(cudaFuncSetAttribute(k_line_part<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    FV_CUDA(cudaFuncSetAttribute(k_line_part<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    done = true;
  }
  return FV_OK;
}

// a launch, timed under `kind` by the grid's profiler and counted
#define MG_LAUNCH(kind, ...)          \
  do {                                \
    LaunchScope ls_(g, kind);         \
    __VA_ARGS__;                      \
    FV_CHECK_LAUNCH();                \
  } while (0)

// one V-cycle on level l: lev[l].b -> lev[l].x[cur] (zero start)
fv_status vcycle(const fv_grid* g, MgState* M, int l, int nu, float omega, cudaStream_t st) {
  MgLevelHost& H = M->lev[l];
  const LevDev& L = H.dev;
  if (l == M->nlev - 1) {
    MG_LAUNCH(FV_K_MG_OTHER, k_coarse<<<1, 64, 0, st>>>(M->coarse, H.b, H.x[0]));
    H.cur = 0;
    return FV_OK;
  }
  FV_CUDA(cudaMemsetAsync(H.x[0], 0, L.ncell * sizeof(float), st));
  float* x = H.x[0];
  auto sweep = [&](int D, int color) -> fv_status {
    const int na = D == 0 ? L.n[1] : L.n[0];
    const int nb = D == 2 ? L.n[1] : L.n[2];
    const int64_t nlines = (int64_t)((na + 1) / 2) * nb;
    const int nl = L.n[D];
    if (nl <= kPartMaxLine) {     // lines split over P warps, 32 lines per block
      // segments of >= 4 rows: short chains on the coarse levels too
      const int P = std::max(1, std::min(8, nl / 4));
      const int nblk = (int)((nlines + 31) / 32);
      const size_t sm = part_smem(nl, P);
      if (D == 0) MG_LAUNCH(FV_K_MG_SMOOTH, k_line_part<0><<<nblk, 32 * P, sm, st>>>(L, x, H.b, omega, color, P));
      else if (D == 1) MG_LAUNCH(FV_K_MG_SMOOTH, k_line_part<1><<<nblk, 32 * P, sm, st>>>(L, x, H.b, omega, color, P));
      else MG_LAUNCH(FV_K_MG_SMOOTH, k_line_part<2><<<nblk, 32 * P, sm, st>>>(L, x, H.b, omega, color, P));
      return FV_OK;
    }
    const int nblk = (int)((nlines + 127) / 128);
    if (D == 0) MG_LAUNCH(FV_K_MG_SMOOTH, k_line<0><<<nblk, 128, 0, st>>>(L, x, H.b, H.cb, H.db, omega, color));
    else if (D == 1) MG_LAUNCH(FV_K_MG_SMOOTH, k_line<1><<<nblk, 128, 0, st>>>(L, x, H.b, H.cb, H.db, omega, color));
    else MG_LAUNCH(FV_K_MG_SMOOTH, k_line<2><<<nblk, 128, 0, st>>>(L, x, H.b, H.cb, H.db, omega, color));
    return FV_OK;
  };
  // symmetric Gauss-Seidel: x, y, z (colours 0, 1) before, the exact reverse after
  for (int s = 0; s < nu; ++s)
    for (int D = 0; D < 3; ++D)
      for (int c = 0; c < 2; ++c) FV_TRY(sweep(D, c));
  const MgLevelHost& C = M->lev[l + 1];
  MG_LAUNCH(FV_K_MG_OTHER, k_resid32<<<blocks_for(L.ncell), 256, 0, st>>>(L, x, H.b, H.res));
  MG_LAUNCH(FV_K_MG_OTHER, k_restrict<<<blocks_for(C.dev.ncell), 256, 0, st>>>(L, C.dev.n[0], C.dev.n[1], C.dev.n[2], H.res,
                                                    C.b));
  FV_TRY(vcycle(g, M, l + 1, nu, omega, st));
  MG_LAUNCH(FV_K_MG_OTHER, k_prolong_add<<<blocks_for(L.ncell), 256, 0, st>>>(L, C.dev.n[0], C.dev.n[1], C.x[C.cur],
                                                     x));
  for (int s = 0; s < nu; ++s)
    for (int D = 2; D >= 0; --D)
      for (int c = 1; c >= 0; --c) FV_TRY(sweep(D, c));
  H.cur = 0;
  return FV_OK;
}

// z = M^-1 r: round r into level 0, one V-cycle, widen
fv_status precondition(fv_grid* g, MgState* M, const double* r, double* z, int nu, float omega) {
  cudaStream_t st = g->stream;
  FV_TRY(set_part_attributes());
  MgLevelHost& H = M->lev[0];
  MG_LAUNCH(FV_K_MG_OTHER, k_round_cells<<<blocks_for(g->ncell), 256, 0, st>>>(g->ncell, r, H.b));
  FV_TRY(vcycle(g, M, 0, nu, omega, st));
  MG_LAUNCH(FV_K_MG_OTHER, k_widen_cells<<<blocks_for(g->ncell), 256, 0, st>>>(g->ncell, H.x[H.cur], z));
  return FV_OK;
}

}  // namespace

void destroy_mg(fv_grid* g) {
  MgState* M = (MgState*)g->mg;
  if (!M) return;
  if (M->d_tab) cudaFree(M->d_tab);
  if (M->d_work) cudaFree(M->d_work);
  if (M->r) cudaFree(M->r);
  if (M->h_s) cudaFreeHost(M->h_s);
  delete M;
  g->mg = nullptr;
}

fv_status mg_solve(fv_grid* g, const double* r, double* phi, const double* guess,
                   const fv_mg_opts& o, fv_mg_stats* stats) {
  if (!g->mg) {
    const fv_status s = build_mg(g);
    if (s != FV_OK) {
      destroy_mg(g);
      return s;
    }
  }
  MgState* M = (MgState*)g->mg;
  cudaStream_t st = g->stream;
  const int64_t n = g->ncell;
  const int nb = kRedBlocks;
  fv_mg_stats sv = {};
  sv.levels = M->nlev;
  // compatible right-hand side and the initial residual
  MG_LAUNCH(FV_K_MG_OTHER, k_sum_vr<<<nb, kRedThreads, 0, st>>>(M->fine, r, M->part));
  MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_STORE, S_VR, 0, M->s));
  if (guess && guess != phi)
    FV_CUDA(cudaMemcpyAsync(phi, guess, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (!guess) FV_CUDA(cudaMemsetAsync(phi, 0, n * sizeof(double), st));
  MG_LAUNCH(FV_K_MG_OTHER, k_rhs<<<nb, kRedThreads, 0, st>>>(M->fine, r, M->s, M->vtot, guess ? phi : nullptr, M->r,
                                     M->part));
  MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_STORE, S_BB, 0, M->s));
  // the initial residual norm (guess given) for the convergence test
  MG_LAUNCH(FV_K_MG_OTHER, k_dots2<<<nb, kRedThreads, 0, st>>>(n, M->r, M->r, M->r, M->part));
  MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_BETA, 0, 1, M->s));
  FV_CUDA(cudaMemcpyAsync(M->h_s, M->s, S_N * sizeof(double), cudaMemcpyDeviceToHost, st));
  FV_CUDA(cudaStreamSynchronize(st));
  const double bnorm = std::sqrt(M->h_s[S_BB]);
  double rnorm = std::sqrt(std::max(M->h_s[S_RZ], 0.0));
  const float omega = (float)o.omega;
  int it = 0, zc = 0;
  if (bnorm > 0.0 && std::isfinite(rnorm)) {
    while (rnorm > o.rtol * bnorm && it < o.max_iter) {
      double* z = M->z[zc];
      double* zo = M->z[zc ^ 1];
      FV_TRY(precondition(g, M, M->r, z, o.nu, omega));
      if (it == 0) FV_CUDA(cudaMemsetAsync(zo, 0, n * sizeof(double), st));
      MG_LAUNCH(FV_K_MG_OTHER, k_dots2<<<nb, kRedThreads, 0, st>>>(n, M->r, z, zo, M->part));
      MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_BETA, 0, it == 0, M->s));
      MG_LAUNCH(FV_K_MG_OTHER, k_cg_dir<<<blocks_for(n), 256, 0, st>>>(n, M->s, z, M->p));
      MG_LAUNCH(FV_K_MG_OTHER, k_apply64<<<nb, kRedThreads, 0, st>>>(M->fine, M->p, M->q, M->part));
      MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_ALPHA, 0, 0, M->s));
      MG_LAUNCH(FV_K_MG_OTHER, k_cg_step<<<nb, kRedThreads, 0, st>>>(n, M->s, M->p, M->q, phi, M->r, M->part));
      MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_STORE, S_RR, 0, M->s));
      FV_CUDA(cudaMemcpyAsync(M->h_s, M->s, S_N * sizeof(double), cudaMemcpyDeviceToHost, st));
      FV_CUDA(cudaStreamSynchronize(st));
      ++it;
      zc ^= 1;
      rnorm = std::sqrt(std::max(M->h_s[S_RR], 0.0));
      if (!std::isfinite(rnorm)) break;
    }
  }
  // zero volume-weighted mean
  MG_LAUNCH(FV_K_MG_OTHER, k_sum_vr<<<nb, kRedThreads, 0, st>>>(M->fine, phi, M->part));
  MG_LAUNCH(FV_K_MG_OTHER, k_finalize<<<1, kRedThreads, 0, st>>>(M->part, nb, OP_STORE, S_VPHI, 0, M->s));
  MG_LAUNCH(FV_K_MG_OTHER, k_sub_mean<<<blocks_for(n), 256, 0, st>>>(n, M->s, M->vtot, phi));
  sv.iterations = it;
  sv.rel_res = bnorm > 0.0 ? rnorm / bnorm : 0.0;
  if (stats) *stats = sv;
  if (!std::isfinite(rnorm)) {
    set_error("fv_pressure_solve_mg: NaN in the residual");
    return FV_ENAN;
  }
  if (bnorm > 0.0 && rnorm > o.rtol * bnorm) {
    set_error("fv_pressure_solve_mg: no convergence within max_iter");
    return FV_ENOCONV;
  }
  return FV_OK;
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_pressure_solve_mg(fv_grid* g, const double* r, double* phi,
                                          const double* guess, const fv_mg_opts* opts,
                                          fv_mg_stats* stats) {
  if (!g || !r || !phi) {
    set_error("fv_pressure_solve_mg: NULL argument");
    return FV_EINVAL;
  }
  fv_mg_opts o = {};
  if (opts) o = *opts;
  if (o.rtol <= 0) o.rtol = 1e-10;
  if (o.max_iter <= 0) o.max_iter = 100;
  if (o.nu <= 0) o.nu = 1;
  if (o.omega <= 0) o.omega = 1.0;
  if (o.nu > 8 || o.omega >= 2.0) {
    set_error("fv_pressure_solve_mg: bad option (nu <= 8, 0 < omega < 2)");
    return FV_EINVAL;
  }
  return mg_solve(g, r, phi, guess, o, stats);
}

// host-only: the 1-D multigrid hierarchy of one axis
extern "C" int fv_host_mg_axis(int n, int map, int level, int* n_out, double* faces,
                               int* pc0, double* pw1) {
  if (n < 1 || level < 0 || !n_out || map < 0 || map > 2) return FV_EINVAL;
  std::vector<Axis1D> ax;
  ax.push_back(axis_from_faces(map_faces(n, map)));
  for (int l = 0; l < level; ++l) ax.push_back(coarsen(ax.back()));
  const Axis1D& a = ax[level];
  *n_out = a.n;
  if (faces) std::memcpy(faces, a.x.data(), (a.n + 1) * sizeof(double));
  if (pc0 || pw1) {
    const Axis1D c = coarsen(a);
    std::vector<int> c0;
    std::vector<double> w1;
    prolongation(a, c, c0, w1);
    if (pc0) std::memcpy(pc0, c0.data(), a.n * sizeof(int));
    if (pw1) std::memcpy(pw1, w1.data(), a.n * sizeof(double));
  }
  return FV_OK;
}

extern "C" int fv_host_mg_levels(int nx, int ny, int nz) {
  const int n[3] = {nx, ny, nz};
  if (nx < 1 || ny < 1 || nz < 1) return -1;
  return count_levels(n);
}
