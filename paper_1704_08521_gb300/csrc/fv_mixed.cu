// Mixed-precision SIMPLE loop (Section 3, the algorithm after Eq. 10) laid
// out for GB300, whose FP64 pipes run at ~1/70 of the FP32 rate:
//   * J.v and the pressure-correction transforms in float32;
//   * the velocity/pressure state of the loop as float-float pairs
//     (hi + lo, ~48 bits), updated and differenced on the FP32 pipes, so the
//     divergence that drives the next correction is computed far below
//     float32 round-off (the defect-correction residual);
//   * float64 only at the API boundary, converted with integer operations.
// Each pass reads/writes every field once: the correction of the cell's own
// faces, the on-the-fly correction of its high faces and the new divergence
// are fused in one kernel (ping-pong buffers, no read-after-write hazard).
#include "fv_ff.cuh"
#include "fv_internal.cuh"
#include "fv_stencil_dev.cuh"
#include "fv_tc5.cuh"
#include "fv_jv.cuh"

namespace fv {

namespace {

__device__ __forceinline__ float2 to2(ff a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ ff of2(float2 a) { return {a.x, a.y}; }

__device__ __forceinline__ float block_maxf(float v) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < nw) ? red[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

__global__ void k_round_f32(const double* __restrict__ in, float* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = f64_round_f32(__ldg(in + e));
}

__global__ void k_widen_f32(const float* __restrict__ in, double* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = f32_to_f64(__ldg(in + e));
}

// D w in float32 (first residual of the loop; w holds float32 values).
__global__ void __launch_bounds__(256) k_div_f32(MetFF m, const float* __restrict__ w,
                                                 float* __restrict__ r) {
  tc5::pdl_trigger();   // the pressure transform that follows may start its set-up
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  if (!act_) return;
  for (int kk = 0; kk < kCellKz; ++kk) {
  const int k = blockIdx.y * kCellKz + kk;
  if (k >= m.n[2]) return;
  const int64_t nx = m.n[0], nxy = nx * m.n[1], nc = m.ncell;
  const int64_t base = ((int64_t)k * m.n[1] + j) * nx + i;
  const float u0 = (i > 0) ? w[base] : 0.f;
  const float u1 = (i + 1 < m.n[0]) ? w[base + 1] : 0.f;
  const float v0 = (j > 0) ? w[nc + base] : 0.f;
  const float v1 = (j + 1 < m.n[1]) ? w[nc + base + nx] : 0.f;
  const float w0 = (k > 0) ? w[2 * nc + base] : 0.f;
  const float w1 = (k + 1 < m.n[2]) ? w[2 * nc + base + nxy] : 0.f;
  r[base] = (u1 - u0) * m.idx[0][i].x + (v1 - v0) * m.idx[1][j].x + (w1 - w0) * m.idx[2][k].x;
  }
}

// One pass: v_out = v_in - omega G phi (own faces), p += omega phi, and
// r = D v_out in float-float arithmetic, rounded to float32 for the next
// pressure-correction solve.  FIRST: v_in is the float32 predictor w.
template <bool FIRST, bool FFG = false>
__global__ void __launch_bounds__(256) k_correct_ff(MetFF m, const void* __restrict__ vin_,
                                                    float2* __restrict__ vout,
                                                    const float* __restrict__ phi,
                                                    float2* __restrict__ p, float* __restrict__ r,
                                                    float omega, double* scal) {
  tc5::pdl_trigger();   // the pressure transform that follows may start its set-up
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  float aphi = 0.f, adiv = 0.f;
  for (int kk = 0; kk < kCellKz; ++kk) {
    const int k = blockIdx.y * kCellKz + kk;
    if (!act_ || k >= m.n[2]) continue;
    const int pos[3] = {i, j, k};
    const int st[3] = {1, m.n[0], m.n[0] * m.n[1]};
    const int nc = (int)m.ncell;
    const int base = (k * m.n[1] + j) * m.n[0] + i;
    const float* w32 = (const float*)vin_;
    const float2* vin = (const float2*)vin_;
    auto load = [&](int e) -> ff {
      if (FIRST) return {__ldg(w32 + e), 0.f};
      return of2(__ldg(vin + e));
    };
    const float f0 = __ldg(phi + base);
    ff dv = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = pos[c];
      ff lo = {0.f, 0.f}, hi = {0.f, 0.f};
      if (q > 0) {
        if (FFG) {   // gradient of the float32 phi evaluated in float-float
          const ff gr = ff_mul(two_sum(f0, -__ldg(phi + base - st[c])), of2(m.idcf[c][q]));
          lo = ff_sub(load(c * nc + base), ff_mul_f(gr, omega));
        } else {
          const float g = (f0 - __ldg(phi + base - st[c])) * m.idc[c][q];
          lo = ff_add_f(load(c * nc + base), -omega * g);
        }
      }
      vout[c * nc + base] = to2(lo);
      if (q + 1 < m.n[c]) {
        if (FFG) {
          const ff gr = ff_mul(two_sum(__ldg(phi + base + st[c]), -f0), of2(m.idcf[c][q + 1]));
          hi = ff_sub(load(c * nc + base + st[c]), ff_mul_f(gr, omega));
        } else {
          const float g = (__ldg(phi + base + st[c]) - f0) * m.idc[c][q + 1];
          hi = ff_add_f(load(c * nc + base + st[c]), -omega * g);
        }
      }
      dv = ff_add(dv, ff_mul(ff_sub(hi, lo), of2(m.idx[c][q])));
    }
    r[base] = dv.hi;
    if (FIRST) p[base] = make_float2(omega * f0, 0.f);
    else p[base] = to2(ff_add_f(of2(p[base]), omega * f0));
    const float a1 = fabsf(f0), a2 = fabsf(dv.hi);
    if (!(a1 <= 3e38f) || !(a2 <= 3e38f)) scal[S_NAN] = 1.0;
    else { aphi = fmaxf(aphi, a1); adiv = fmaxf(adiv, a2); }
  }
  aphi = block_maxf(aphi);
  adiv = block_maxf(adiv);
  if (threadIdx.x == 0) {
    atomicMax((unsigned*)(scal + S_PHI_MAX_F), __float_as_uint(aphi));
    atomicMax((unsigned*)(scal + S_DIV_MAX_F), __float_as_uint(adiv));
  }
}

__global__ void k_join_ff(const float2* __restrict__ v, const double* __restrict__ x, float sigma,
                          double* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    ff a = of2(__ldg(v + e));
    if (x) a = ff_sub(a, ff_mul_f(f64_split(__ldg(x + e)), sigma));
    out[e] = ff_join(a.hi, a.lo);
  }
}

// FV_FF operands: exact float-float split of float64 values
__global__ void k_split_ff(const double* __restrict__ in, float2* __restrict__ out, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = to2(f64_split(__ldg(in + e)));
}

// D w of a float-float field, rounded to float32 (first pressure rhs of FV_FF)
__global__ void __launch_bounds__(256) k_div_ff(MetFF m, const float2* __restrict__ w,
                                                float* __restrict__ r) {
  tc5::pdl_trigger();   // the pressure transform that follows may start its set-up
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  if (t_ >= plane_) return;
  const int i = t_ % m.n[0], j = t_ / m.n[0];
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int nc = (int)m.ncell;
  for (int kk = 0; kk < kCellKz; ++kk) {
    const int k = blockIdx.y * kCellKz + kk;
    if (k >= nz) return;
    const int base = k * plane_ + t_;
    const ff z = {0.f, 0.f};
    const ff u0 = (i > 0) ? of2(w[base]) : z, u1 = (i + 1 < nx) ? of2(w[base + 1]) : z;
    const ff v0 = (j > 0) ? of2(w[nc + base]) : z, v1 = (j + 1 < ny) ? of2(w[nc + base + nx]) : z;
    const ff w0 = (k > 0) ? of2(w[2 * nc + base]) : z;
    const ff w1 = (k + 1 < nz) ? of2(w[2 * nc + base + plane_]) : z;
    ff d = ff_mul(ff_sub(u1, u0), of2(m.idx[0][i]));
    d = ff_add(d, ff_mul(ff_sub(v1, v0), of2(m.idx[1][j])));
    d = ff_add(d, ff_mul(ff_sub(w1, w0), of2(m.idx[2][k])));
    r[base] = d.hi;
  }
}

inline unsigned grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

inline dim3 cell_grid(const fv_grid* g, int) { return cell_launch_grid(g->n); }

inline int block_x(const fv_grid*) { return kCellThreads; }

}  // namespace

fv_status launch_round_f32(const fv_grid* g, const double* in, float* out, int64_t n) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_round_f32<<<grid1d(n), 256, 0, g->stream>>>(in, out, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_widen_f32(const fv_grid* g, const float* in, double* out, int64_t n) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_widen_f32<<<grid1d(n), 256, 0, g->stream>>>(in, out, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_div_f32(const fv_grid* g, const float* w32, float* r32) {
  const int bx = block_x(g);
  {
    LaunchScope ls_(g, FV_K_DIVERGENCE);
    k_div_f32<<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_ff, w32, r32);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_correct_ff(const fv_grid* g, bool first, const void* vin, float2* vout,
                            const float* phi, float2* p, float* r, double omega, bool ffg) {
  const int bx = block_x(g);
  {
    LaunchScope ls_(g, FV_K_CORRECT);
    if (first)
      k_correct_ff<true><<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_ff, vin, vout, phi, p, r,
                                                                 float(omega), g->d_scal);
    else if (ffg)
      k_correct_ff<false, true><<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_ff, vin, vout, phi, p,
                                                                        r, float(omega), g->d_scal);
    else
      k_correct_ff<false><<<cell_grid(g, bx), bx, 0, g->stream>>>(g->met_ff, vin, vout, phi, p, r,
                                                                  float(omega), g->d_scal);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_join_ff(const fv_grid* g, const float2* v, const double* x, double sigma,
                         double* out, int64_t n) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_join_ff<<<grid1d(n), 256, 0, g->stream>>>(v, x, float(sigma), out, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_split_ff(const fv_grid* g, const double* in, float2* out, int64_t n) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_split_ff<<<grid1d(n), 256, 0, g->stream>>>(in, out, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

// float-float J.v (FV_FF): U from Ud (float64, split into g->Uff first,
// which drops a registered base flow) or, when Ud is null, from the grid's
// registered base flow g->Uff; x float64 split as its planes are staged;
// float-float result (this file is compiled without FMA contraction, so
// every TwoSum and TwoProd keeps its rounding)
fv_status launch_jv_ff(const fv_grid* g, const double* Ud, const double* x, float2* out,
                       double shift, const void* call) {
  if (Ud) {
    FV_TRY(launch_split_ff(g, Ud, g->Uff, g->nvel));
    const_cast<fv_grid*>(g)->base_ptr = nullptr;
  }
  jv::Args<ffn, float2, float2> a;
  a.m = g->met_fn;
  a.Ur = g->Uff;
  a.x = x;
  a.out = out;
  a.call = (const jv::CallPtrs*)call;
  a.inv_re = ffn(f64_split(1.0 / g->re));
  a.shift = ffn(f64_split(shift));
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    FV_CUDA(jv::launch(a, g->stream));
  }
  return FV_OK;
}

fv_status launch_jv_ff_out64(const fv_grid* g, const double* Ud, const double* x, double* out,
                             double shift) {
  if (Ud) {
    FV_TRY(launch_split_ff(g, Ud, g->Uff, g->nvel));
    const_cast<fv_grid*>(g)->base_ptr = nullptr;
  }
  jv::Args<ffn, float2, double> a;
  a.m = g->met_fn;
  a.Ur = g->Uff;
  a.x = x;
  a.out = out;
  a.call = nullptr;
  a.inv_re = ffn(f64_split(1.0 / g->re));
  a.shift = ffn(f64_split(shift));
  {
    LaunchScope ls_(g, FV_K_MOMENTUM);
    FV_CUDA(jv::launch(a, g->stream));
  }
  return FV_OK;
}

fv_status launch_div_ff(const fv_grid* g, const float2* w, float* r32) {
  {
    LaunchScope ls_(g, FV_K_DIVERGENCE);
    k_div_ff<<<cell_grid(g, 0), kCellThreads, 0, g->stream>>>(g->met_ff, w, r32);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status set_base(fv_grid* g, const double* U) {
  FV_TRY(launch_round_f32(g, U, g->U32, g->nvel));
  FV_TRY(launch_split_ff(g, U, g->Uff, g->nvel));
  g->base_ptr = U;
  return FV_OK;
}

fv_status launch_join_ff_cells(const fv_grid* g, const float2* p, double* out) {
  return launch_join_ff(g, p, nullptr, 0.0, out, g->ncell);
}

}  // namespace fv
