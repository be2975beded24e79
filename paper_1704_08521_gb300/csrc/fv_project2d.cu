// Divergence-free projections of a velocity field onto coordinate planes and
// their vector potentials (Section 4, Eqs. 11-17), in float64.
//
// For the planes (a, c) with normal direction b the projection keeps the two
// in-plane components, sets the normal one to zero and removes the part that
// is not divergence-free in the plane (Eqs. 12-14): plane by plane, the
// two-dimensional Leray projection  v_b = q - G_ac phi  with
// (L_a (+) L_c) phi = D_ac q  (Neumann walls, phi of zero mean in every
// plane), solved exactly by the eigenbases of the pressure operator along a
// and c: two forward transforms, division by lam_a + lam_c (the plane's
// constant null mode set to zero), two inverse transforms.  With this exact
// solve the paper's 2-D SIMPLE-like loop ends after its first correction.
// The vector potential (Eqs. 15-17) has the single component Psi^(b) on the
// corners of the plane's cells, zero on the walls: the running integral
// along a of the in-plane component c,
//   (x, z): Psi_{i+1} = Psi_i + w dx_i     (w = dPsi/dx, u = -dPsi/dz)
//   (y, z): Psi_{j+1} = Psi_j - w dy_j     (w = -dPsi/dy, v = dPsi/dz)
//   (x, y): Psi_{i+1} = Psi_i - v dx_i     (v = -dPsi/dx, u = dPsi/dy)
#include "fv_internal.cuh"

namespace fv {

namespace {

constexpr int kPlaneA[3] = {0, 1, 0}, kPlaneC[3] = {2, 2, 1}, kPlaneB[3] = {1, 0, 2};

__device__ __forceinline__ void cell_of(int64_t e, const int n[3], int (&p)[3]) {
  p[0] = (int)(e % n[0]);
  p[1] = (int)((e / n[0]) % n[1]);
  p[2] = (int)(e / ((int64_t)n[0] * n[1]));
}

// r = D_ac q (the in-plane divergence; wall faces read as zero)
__global__ void k_div2d(Met<double> m, const double* __restrict__ q, int a, int c, double* __restrict__ r) {
  const int64_t nc = m.ncell;
  const int64_t st[3] = {1, m.n[0], (int64_t)m.n[0] * m.n[1]};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    int p[3];
    cell_of(e, m.n, p);
    double s = 0.0;
    const int ds[2] = {a, c};
    for (int t = 0; t < 2; ++t) {
      const int d = ds[t];
      const double lo = p[d] > 0 ? q[d * nc + e] : 0.0;
      const double hi = p[d] + 1 < m.n[d] ? q[d * nc + e + st[d]] : 0.0;
      s += (hi - lo) * m.idx[d][p[d]];
    }
    r[e] = s;
  }
}

// hat /= lam_a + lam_c; the constant mode of each plane -> 0
__global__ void k_scale2d(TpfDev<double> tp, int a, int c, double* __restrict__ h, int64_t ncell) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ncell;
       e += (int64_t)gridDim.x * blockDim.x) {
    int p[3];
    cell_of(e, tp.n, p);
    if (p[a] == tp.null_index[a] && p[c] == tp.null_index[c]) h[e] = 0.0;
    else h[e] = h[e] / (tp.lam[a][p[a]] + tp.lam[c][p[c]]);
  }
}

// vp = q - G_ac phi on the in-plane components (walls zero), vp_b = 0
__global__ void k_correct2d(Met<double> m, const double* __restrict__ q, const double* __restrict__ phi,
                            int a, int c, double* __restrict__ vp) {
  const int64_t nc = m.ncell;
  const int64_t st[3] = {1, m.n[0], (int64_t)m.n[0] * m.n[1]};
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nc;
       e += (int64_t)gridDim.x * blockDim.x) {
    int p[3];
    cell_of(e, m.n, p);
    for (int d = 0; d < 3; ++d) {
      double v = 0.0;
      if ((d == a || d == c) && p[d] > 0)
        v = q[d * nc + e] - (phi[e] - phi[e - st[d]]) * m.idc[d][p[d]];
      vp[d * nc + e] = v;
    }
  }
}

// Psi on the corners: one thread per line along a (index b, c-corner k)
__global__ void k_potential(Met<double> m, const double* __restrict__ vp, int a, int c, int b, double sgn,
                            double* __restrict__ psi) {
  const int nb = m.n[b], ncp = m.n[c] + 1, nap = m.n[a] + 1;
  const int64_t lines = (int64_t)nb * ncp;
  const int64_t nc = m.ncell;
  const int64_t st[3] = {1, m.n[0], (int64_t)m.n[0] * m.n[1]};
  // strides of the corner array: [z][y][x] with n + 1 along a and c
  int64_t cs[3];
  {
    int64_t dims[3] = {m.n[0], m.n[1], m.n[2]};
    dims[a] += 1;
    dims[c] += 1;
    cs[0] = 1;
    cs[1] = dims[0];
    cs[2] = dims[0] * dims[1];
  }
  for (int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; l < lines;
       l += (int64_t)gridDim.x * blockDim.x) {
    const int jb = (int)(l % nb), kc = (int)(l / nb);
    double s = 0.0;
    int64_t o = jb * cs[b] + kc * cs[c];
    psi[o] = 0.0;
    for (int ia = 0; ia < nap - 1; ++ia) {
      // component c on c-face kc (face n_c is the wall: zero), centre ia
      double comp = 0.0;
      if (kc < m.n[c]) comp = vp[c * nc + (int64_t)ia * st[a] + (int64_t)jb * st[b] + (int64_t)kc * st[c]];
      s += sgn * comp * m.dx[a][ia];
      psi[o + (int64_t)(ia + 1) * cs[a]] = kc < m.n[c] ? s : 0.0;
    }
  }
}

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

fv_status plane_projection(const fv_grid* g, const double* v, int plane, double* vp, double* psi) {
  const int a = kPlaneA[plane], c = kPlaneC[plane], b = kPlaneB[plane];
  double* r = g->cell_buf[0];
  double* t0 = (double*)g->tpf_buf[0];
  double* t1 = (double*)g->tpf_buf[1];
  {
    LaunchScope ls_(g, FV_K_DIVERGENCE);
    k_div2d<<<blocks_for(g->ncell), 256, 0, g->stream>>>(g->met_d, v, a, c, r);
  }
  FV_CHECK_LAUNCH();
  FV_TRY(transform_axis_f64(g, a, g->tpf_d.Einv[a], r, t0));
  FV_TRY(transform_axis_f64(g, c, g->tpf_d.Einv[c], t0, t1));
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_scale2d<<<blocks_for(g->ncell), 256, 0, g->stream>>>(g->tpf_d, a, c, t1, g->ncell);
  }
  FV_CHECK_LAUNCH();
  FV_TRY(transform_axis_f64(g, c, g->tpf_d.E[c], t1, t0));
  FV_TRY(transform_axis_f64(g, a, g->tpf_d.E[a], t0, r));   // r = phi
  {
    LaunchScope ls_(g, FV_K_CORRECT);
    k_correct2d<<<blocks_for(g->ncell), 256, 0, g->stream>>>(g->met_d, v, r, a, c, vp);
  }
  FV_CHECK_LAUNCH();
  if (psi) {
    const double sgn = plane == 0 ? 1.0 : -1.0;
    const int64_t lines = (int64_t)g->n[b] * (g->n[c] + 1);
    LaunchScope ls_(g, FV_K_VECTOR);
    k_potential<<<blocks_for(lines), 256, 0, g->stream>>>(g->met_d, vp, a, c, b, sgn, psi);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

}  // namespace fv

extern "C" fv_status fv_plane_projection(const fv_grid* g, const double* v, int plane, double* vp,
                                         double* psi) {
  if (!g || !v || !vp) { fv::set_error("fv_plane_projection: NULL argument"); return FV_EINVAL; }
  if (plane < 0 || plane > 2) { fv::set_error("fv_plane_projection: plane must be 0, 1 or 2"); return FV_EINVAL; }
  if (v == vp) { fv::set_error("fv_plane_projection: v and vp alias"); return FV_EINVAL; }
  return fv::plane_projection(g, v, plane, vp, psi);
}
