// Right preconditioner of the Newton corrections: M^-1 y = P (s - Lap/Re)^-1 y.
//
// Section 3 solves the Newton correction J u = F with GMRES / BiCGstab(2)
// whose Krylov vectors are the SIMPLE projections P L_U v (Eqs. 8-10), with
// no preconditioner.  On the strongly stretched cosine grids of the
// benchmark configurations the diffusive part of L_U spans ~1e7 (the
// smallest cell is ~pi^2 / (4 N^2)), and the unpreconditioned iteration
// counts grow like N^2.  The correction itself does not depend on how it is
// found, so newton_steady optionally applies this Stokes-type right
// preconditioner (flexible GMRES): the inverse of the shifted vector
// Laplacian of the momentum equations, followed by the projection onto
// divergence-free fields, removes the grid-size-dependent stiffness.
//
// The vector Laplacian of the staggered scheme (the diffusion of Eq. 2 with
// homogeneous wall values) is separable per velocity component c: along c
// the 1-D operator acts on the interior faces (the wall faces carry zero
// normal velocity), along the other two axes on the cell-centred values with
// the wall at half a cell.  Each 1-D operator is W^-1 T with T symmetric
// tridiagonal and W the control-volume widths, diagonalised once on the host
// (as the pressure operator's); the solve is the float32 tensor-product
// transform path with the eigenvalue scaling 1 / (s - (lam_x + lam_y + lam_z) / Re).
// The projection runs the mixed-precision SIMPLE loop (float32 pressure
// solves, float-float state) to a relative correction of 1e-7.
#include <cmath>
#include <vector>

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {

namespace {

// 1-D operator of one axis with n cells.  face: unknowns on faces 1..n-1
// (index 0 is the wall: kept as an identity row with a huge eigenvalue, so
// that its value maps to zero); cell: unknowns on cells 0..n-1.
// E (n x n, row = point, column = mode), Einv (row = mode, column = point).
void helm_axis(const std::vector<double>& dx, const std::vector<double>& dc, bool face,
               std::vector<double>& E, std::vector<double>& Einv, std::vector<double>& lam) {
  const int n = (int)dx.size();
  E.assign((size_t)n * n, 0.0);
  Einv.assign((size_t)n * n, 0.0);
  lam.assign(n, 0.0);
  const int off = face ? 1 : 0;
  const int m = n - off;
  std::vector<double> w(m), d(m), e(m > 1 ? m - 1 : 1, 0.0);
  for (int k = 0; k < m; ++k) {
    if (face) {
      const int f = k + 1;   // interior face between cells f - 1 and f
      w[k] = dc[f];
      d[k] = -(1.0 / dx[f] + 1.0 / dx[f - 1]);
      if (k + 1 < m) e[k] = 1.0 / dx[f];
    } else {
      w[k] = dx[k];
      d[k] = -(1.0 / dc[k + 1] + 1.0 / dc[k]);
      if (k + 1 < m) e[k] = 1.0 / dc[k + 1];
    }
  }
  for (int k = 0; k < m; ++k) d[k] /= w[k];
  for (int k = 0; k + 1 < m; ++k) e[k] /= std::sqrt(w[k] * w[k + 1]);
  std::vector<double> lm, Z;
  if (m > 0) sym_tridiag_eig(m, d, e, lm, Z);
  if (face) {
    E[0] = 1.0;
    Einv[0] = 1.0;
    lam[0] = -1e30;          // the wall "mode": scaled to nothing
  }
  for (int a = 0; a < m; ++a) {
    lam[off + a] = lm[a];
    for (int k = 0; k < m; ++k) {
      const double s = std::sqrt(w[k]);
      E[(size_t)(off + k) * n + off + a] = Z[(size_t)k * m + a] / s;
      Einv[(size_t)(off + a) * n + off + k] = Z[(size_t)k * m + a] * s;
    }
  }
}

fv_status build_tables(fv_grid* g) {
  size_t total = 0;
  for (int d = 0; d < 3; ++d) total += 2 * (2 * (size_t)g->n[d] * g->n[d]) + 3 * (size_t)g->n[d];
  std::vector<float> h(total, 0.f);
  size_t off_E[3][2], off_I[3][2], off_L[3][3], o = 0;
  for (int d = 0; d < 3; ++d) {
    const int n = g->n[d];
    for (int t = 0; t < 2; ++t) {
      std::vector<double> E, Ei, lam;
      helm_axis(g->h_dx[d], g->h_dc[d], t == 0, E, Ei, lam);
      g->helm_lam[d][t] = lam;
      off_E[d][t] = o;
      for (size_t q = 0; q < E.size(); ++q) h[o + q] = (float)E[q];
      o += E.size();
      off_I[d][t] = o;
      for (size_t q = 0; q < Ei.size(); ++q) h[o + q] = (float)Ei[q];
      o += Ei.size();
    }
    for (int c = 0; c < 3; ++c) { off_L[d][c] = o; o += n; }   // scaled eigenvalues per component
  }
  cudaError_t e = cudaMalloc(&g->d_helm, total * sizeof(float));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    g->d_helm = nullptr;
    set_error("cudaMalloc of the preconditioner tables failed");
    return FV_ENOMEM;
  }
  g->ws_bytes += (int64_t)(total * sizeof(float));
  FV_CUDA(cudaMemcpy(g->d_helm, h.data(), total * sizeof(float), cudaMemcpyHostToDevice));
  const float* base = (const float*)g->d_helm;
  for (int c = 0; c < 3; ++c) {
    TpfDev<float>& tp = g->helm[c];
    for (int d = 0; d < 3; ++d) {
      const int t = d == c ? 0 : 1;
      tp.n[d] = g->n[d];
      tp.null_index[d] = -1;
      tp.E[d] = base + off_E[d][t];
      tp.Einv[d] = base + off_I[d][t];
      tp.lam[d] = base + off_L[d][c];
      tp.Et[d] = nullptr;
      tp.Einvt[d] = nullptr;
    }
  }
  g->helm_sigma = g->helm_re = -1.0;
  return FV_OK;
}

// scaled eigenvalues lam'_d = s / 3 - lam_d / Re (their sum is the
// denominator s - (lam_x + lam_y + lam_z) / Re of the transform scaling)
fv_status set_scaling(fv_grid* g, double sigma_p) {
  if (g->helm_sigma == sigma_p && g->helm_re == g->re) return FV_OK;
  for (int c = 0; c < 3; ++c)
    for (int d = 0; d < 3; ++d) {
      const std::vector<double>& lam = g->helm_lam[d][d == c ? 0 : 1];
      std::vector<float> v(lam.size());
      for (size_t a = 0; a < lam.size(); ++a) v[a] = (float)(sigma_p / 3.0 - lam[a] / g->re);
      FV_CUDA(cudaMemcpyAsync((void*)g->helm[c].lam[d], v.data(), v.size() * sizeof(float),
                              cudaMemcpyHostToDevice, g->stream));
    }
  FV_CUDA(cudaStreamSynchronize(g->stream));   // the host vectors above die here
  g->helm_sigma = sigma_p;
  g->helm_re = g->re;
  return FV_OK;
}

}  // namespace

fv_status stokes_precond_apply(fv_grid* g, const double* y, double* out, double sigma_p) {
  if (!g->d_helm) FV_TRY(build_tables(g));
  FV_TRY(set_scaling(g, sigma_p));
  FV_TRY(launch_round_f32(g, y, g->x32, g->nvel));
  for (int c = 0; c < 3; ++c)
    FV_TRY(tpf_run_f32(g, g->helm[c], g->x32 + c * g->ncell, g->w32 + c * g->ncell));
  FV_TRY(launch_div_f32(g, g->w32, g->r32));
  return simple_project_w32(g, out, 1e-7);
}

void destroy_stokes_tables(fv_grid* g) {
  if (g->d_helm) cudaFree(g->d_helm);
  g->d_helm = nullptr;
}

}  // namespace fv
