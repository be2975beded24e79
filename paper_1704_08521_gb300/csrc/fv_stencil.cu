// Staggered finite-volume stencils (Section 3): the linearised momentum
// operator of Eq. 6 / Eq. 10 (J.v), the steady residual of Eqs. 1-4, the
// divergence (Eq. 1) and the fused SIMPLE correction + divergence pass.
//
// One thread per cell (i, j, k), x fastest, so neighbouring threads read
// neighbouring addresses of every field; the three outputs of a cell are the
// momentum balances of its low x-, y- and z-faces.  The scheme:
//   diffusion  : two-point gradients, half-cell distance to a wall value;
//   convection : flux = (transport velocity) x (transported velocity), each
//                linearly interpolated (distance weighted) to the control-
//                volume face; wall fluxes vanish (zero normal velocity).
#include "fv_ff.cuh"
#include "fv_internal.cuh"
#include "fv_stencil_dev.cuh"
#include "fv_jv.cuh"

namespace fv {

namespace {

using stencil::ld;
using stencil::to_out;
using stencil::momentum_face;

template <typename T, bool JAC, typename TI, typename TO>
__global__ void __launch_bounds__(256) k_momentum(Met<T> m, const TI* __restrict__ U,
                                                  const TI* __restrict__ V,
                                                  const double* __restrict__ P,
                                                  TO* __restrict__ out, T inv_re, T lid_u,
                                                  T lid_v, T shift) {
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  if (!act_) return;
  // the planes unrolled so that their loads are in flight together
#pragma unroll
  for (int kk = 0; kk < kCellKz; ++kk) {
  const int k = blockIdx.y * kCellKz + kk;
  if (k >= m.n[2]) continue;
  const int pos[3] = {i, j, k};
  const int st[3] = {1, m.n[0], m.n[0] * m.n[1]};
  const int base = (k * m.n[1] + j) * m.n[0] + i;
  const int nc = (int)m.ncell;
  // u (x-faces)
  {
    T r = T(0);
    if (i > 0) {
      r = momentum_face<T, 0, JAC, TI>(m, U, V, base, pos, st, inv_re, lid_u, shift);
      if (!JAC) r -= T(__ldg(P + base) - __ldg(P + base - 1)) * m.idc[0][i];
    }
    out[base] = to_out<T, TO>(r);
  }
  // v (y-faces)
  {
    T r = T(0);
    if (j > 0) {
      r = momentum_face<T, 1, JAC, TI>(m, U, V, base, pos, st, inv_re, lid_v, shift);
      if (!JAC) r -= T(__ldg(P + base) - __ldg(P + base - st[1])) * m.idc[1][j];
    }
    out[nc + base] = to_out<T, TO>(r);
  }
  // w (z-faces)
  {
    T r = T(0);
    if (k > 0) {
      r = momentum_face<T, 2, JAC, TI>(m, U, V, base, pos, st, inv_re, T(0), shift);
      if (!JAC) r -= T(__ldg(P + base) - __ldg(P + base - st[2])) * m.idc[2][k];
    }
    out[2 * nc + base] = to_out<T, TO>(r);
  }
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* slot, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax((unsigned long long*)slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < nw) ? red[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// D v (Eq. 1) at every cell; wall faces are read as zero.
__global__ void __launch_bounds__(256) k_divergence(Met<double> m, const double* __restrict__ v,
                                                    double* __restrict__ r, double* maxslot,
                                                    double* nanslot) {
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  double a = 0.0;
  for (int kk = 0; kk < kCellKz; ++kk) {
    const int k = blockIdx.y * kCellKz + kk;
    if (!act_ || k >= m.n[2]) continue;
    const int64_t nx = m.n[0], nxy = nx * m.n[1], nc = m.ncell;
    const int64_t base = ((int64_t)k * m.n[1] + j) * nx + i;
    const double u0 = (i > 0) ? v[base] : 0.0;
    const double u1 = (i + 1 < m.n[0]) ? v[base + 1] : 0.0;
    const double v0 = (j > 0) ? v[nc + base] : 0.0;
    const double v1 = (j + 1 < m.n[1]) ? v[nc + base + nx] : 0.0;
    const double w0 = (k > 0) ? v[2 * nc + base] : 0.0;
    const double w1 = (k + 1 < m.n[2]) ? v[2 * nc + base + nxy] : 0.0;
    const double div = (u1 - u0) * m.idx[0][i] + (v1 - v0) * m.idx[1][j] + (w1 - w0) * m.idx[2][k];
    r[base] = div;
    const double ad = fabs(div);
    if (!(ad <= 1e300)) *nanslot = 1.0;
    else a = fmax(a, ad);
  }
  if (maxslot) {
    a = block_max(a);
    if (threadIdx.x == 0) atomic_max_nonneg(maxslot, a);
  }
}

// One SIMPLE pass after the pressure-correction solve (Section 3, step 2):
// vout = vin - omega G phi on the faces owned by the cell, p += omega phi,
// and the new divergence r = D vout, computed from the corrected high faces
// on the fly (vin and vout are different buffers, so no thread reads a face
// another thread has already overwritten).
template <typename PT>
__global__ void __launch_bounds__(256) k_correct_div(Met<double> m, const double* __restrict__ vin,
                                                     double* __restrict__ vout,
                                                     const PT* __restrict__ phi,
                                                     double* __restrict__ p,
                                                     double* __restrict__ r, double omega,
                                                     double* scal) {
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  double aphi = 0.0, adiv = 0.0;
  for (int kk = 0; kk < kCellKz; ++kk) {
    const int k = blockIdx.y * kCellKz + kk;
    if (!act_ || k >= m.n[2]) continue;
    const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
    const int64_t sy = nx, sz = (int64_t)nx * ny, nc = m.ncell;
    const int64_t base = ((int64_t)k * ny + j) * nx + i;
    const double f0 = double(phi[base]);
    // own (low) faces
    double u0 = 0.0, v0 = 0.0, w0 = 0.0;
    if (i > 0) u0 = vin[base] - omega * (f0 - double(phi[base - 1])) * m.idc[0][i];
    if (j > 0) v0 = vin[nc + base] - omega * (f0 - double(phi[base - sy])) * m.idc[1][j];
    if (k > 0) w0 = vin[2 * nc + base] - omega * (f0 - double(phi[base - sz])) * m.idc[2][k];
    vout[base] = u0;
    vout[nc + base] = v0;
    vout[2 * nc + base] = w0;
    // high faces, corrected on the fly
    double u1 = 0.0, v1 = 0.0, w1 = 0.0;
    if (i + 1 < nx) u1 = vin[base + 1] - omega * (double(phi[base + 1]) - f0) * m.idc[0][i + 1];
    if (j + 1 < ny) v1 = vin[nc + base + sy] - omega * (double(phi[base + sy]) - f0) * m.idc[1][j + 1];
    if (k + 1 < nz) w1 = vin[2 * nc + base + sz] - omega * (double(phi[base + sz]) - f0) * m.idc[2][k + 1];
    const double div = (u1 - u0) * m.idx[0][i] + (v1 - v0) * m.idx[1][j] + (w1 - w0) * m.idx[2][k];
    r[base] = div;
    if (p) p[base] += omega * f0;
    const double a1 = fabs(f0), a2 = fabs(div);
    if (!(a1 <= 1e300) || !(a2 <= 1e300)) scal[S_NAN] = 1.0;
    else { aphi = fmax(aphi, a1); adiv = fmax(adiv, a2); }
  }
  aphi = block_max(aphi);
  __syncthreads();
  adiv = block_max(adiv);
  if (threadIdx.x == 0) {
    atomic_max_nonneg(scal + S_PHI_MAX, aphi);
    atomic_max_nonneg(scal + S_DIV_MAX, adiv);
  }
}

__global__ void k_zero_walls(int nx, int ny, int nz, double* v) {
  const int64_t nc = (int64_t)nx * ny * nz;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // u at i = 0: ny*nz entries; v at j = 0: nx*nz; w at k = 0: nx*ny
  const int64_t a = (int64_t)ny * nz, b = (int64_t)nx * nz, c = (int64_t)nx * ny;
  if (t < a) {
    const int64_t kk = t / ny, jj = t % ny;
    v[(kk * ny + jj) * nx] = 0.0;
  } else if (t < a + b) {
    const int64_t s = t - a, kk = s / nx, ii = s % nx;
    v[nc + kk * ny * (int64_t)nx + ii] = 0.0;
  } else if (t < a + b + c) {
    const int64_t s = t - a - b;
    v[2 * nc + s] = 0.0;
  }
}

inline dim3 cell_grid(const fv_grid* g, int) { return cell_launch_grid(g->n); }

inline int block_x(const fv_grid*) { return kCellThreads; }

}  // namespace

fv_status launch_momentum_jac(const fv_grid* g, const double* U, const double* v, double* out,
                              int prec, double shift) {
  if (prec == FV_MIXED) return launch_jv_f32_out64(g, U, v, out, shift);
  jv::Args<double, double, double> a;
  a.m = g->met_d;
  a.Ur = U;
  a.x = v;
  a.out = out;
  a.call = nullptr;
  a.inv_re = 1.0 / g->re;
  a.shift = shift;
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    FV_CUDA(jv::launch(a, g->stream));
  }
  return FV_OK;
}

// float32 J.v of the mixed form: U from Ud (float64, rounded into g->U32
// first, which drops a registered base flow) or, when Ud is null, from the
// grid's registered base flow g->U32; x float64 rounded as its planes are
// staged; float32 result.  call: graph launches read x from the evaluation's
// device call block (whose U the graph has already rounded into g->U32).
fv_status launch_jv_f32(const fv_grid* g, const double* Ud, const double* x, float* out,
                        double shift, const void* call) {
  if (Ud) {
    FV_TRY(launch_round_f32(g, Ud, g->U32, g->nvel));
    const_cast<fv_grid*>(g)->base_ptr = nullptr;
  }
  jv::Args<float, float, float> a;
  a.m = g->met_f;
  a.Ur = g->U32;
  a.x = x;
  a.out = out;
  a.call = (const jv::CallPtrs*)call;
  a.inv_re = float(1.0 / g->re);
  a.shift = float(shift);
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    FV_CUDA(jv::launch(a, g->stream));
  }
  return FV_OK;
}

fv_status launch_jv_f32_out64(const fv_grid* g, const double* Ud, const double* x, double* out,
                              double shift) {
  if (Ud) {
    FV_TRY(launch_round_f32(g, Ud, g->U32, g->nvel));
    const_cast<fv_grid*>(g)->base_ptr = nullptr;
  }
  jv::Args<float, float, double> a;
  a.m = g->met_f;
  a.Ur = g->U32;
  a.x = x;
  a.out = out;
  a.call = nullptr;
  a.inv_re = float(1.0 / g->re);
  a.shift = float(shift);
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    FV_CUDA(jv::launch(a, g->stream));
  }
  return FV_OK;
}

fv_status launch_residual(const fv_grid* g, const double* U, const double* P, double* Fm,
                          double* Fdiv) {
  const int bx = block_x(g);
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    k_momentum<double, false, double, double><<<cell_grid(g, bx), bx, 0, g->stream>>>(
        g->met_d, U, U, P, Fm, 1.0 / g->re, std::cos(g->alpha), std::sin(g->alpha), 0.0);
  }
  FV_CHECK_LAUNCH();
  if (Fdiv) {
    {
      LaunchScope ls_(g, FV_K_DIVERGENCE);
      k_divergence<<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_d, U, Fdiv, nullptr,
                                                           g->d_scal + S_NAN);
    }
    FV_CHECK_LAUNCH();
  }
  return FV_OK;
}

fv_status launch_divergence(const fv_grid* g, const double* v, double* r, double* maxabs_slot) {
  const int bx = block_x(g);
  {
    LaunchScope ls_(g, FV_K_DIVERGENCE);
    k_divergence<<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_d, v, r, maxabs_slot,
                                                         g->d_scal + S_NAN);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_correct_div(const fv_grid* g, const double* vin, double* vout, const void* phi,
                             bool phi_is_float, double* p, double* r, double omega) {
  const int bx = block_x(g);
  if (phi_is_float)
    {
      LaunchScope ls_(g, FV_K_CORRECT);
      k_correct_div<float><<<cell_grid(g, bx), bx, 0, g->stream>>>(
          g->met_d, vin, vout, (const float*)phi, p, r, omega, g->d_scal);
    }
  else
    {
      LaunchScope ls_(g, FV_K_CORRECT);
      k_correct_div<double><<<cell_grid(g, bx), bx, 0, g->stream>>>(
          g->met_d, vin, vout, (const double*)phi, p, r, omega, g->d_scal);
    }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_zero_walls(const fv_grid* g, double* v) {
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int64_t tot = ny * nz + nx * nz + nx * ny;
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_zero_walls<<<(unsigned)((tot + 255) / 256), 256, 0, g->stream>>>(g->n[0], g->n[1], g->n[2], v);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

}  // namespace fv
