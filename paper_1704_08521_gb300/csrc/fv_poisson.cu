// Pressure-correction solve of Section 3, step 1: D G phi = r with
// d phi/dn = 0, by tensor-product factorisation (the paper's TPF method).
// D G = L_x (+) L_y (+) L_z with L = E diag(lam) E^{-1} per axis, so
//   phi = (E_z (x) E_y (x) E_x) diag(1/(lam_x+lam_y+lam_z)) (E_z^-1 (x) E_y^-1 (x) E_x^-1) r
// with the single null mode (constant phi) set to zero.  Each 1-D transform
// is a dense contraction over one axis of the nz x ny x nx array, done by a
// register-tiled shared-memory kernel (64 x 64 outputs per block, 4 x 4 per
// thread); the eigenvalue scaling is fused into the epilogue of the third
// forward transform.  float32 in the mixed mode, float64 otherwise.
#include "fv_internal.cuh"

namespace fv {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

// out[b][p][q] = sum_m M[p][m] in[b][m][q]   (P = K = n; Q columns; B batches)
// SCALE: multiply by 1/(lam_p + lam_y[q / nx] + lam_x[q % nx]), null mode -> 0
template <typename T, typename TI, typename TO, bool SCALE>
__global__ void __launch_bounds__(256) k_left(const T* __restrict__ M, const TI* __restrict__ in,
                                              TO* __restrict__ out, int n, int64_t Q,
                                              TpfDev<T> tp) {
  __shared__ T Ms[TK][TM + 1];
  __shared__ T Is[TK][TN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int p0 = blockIdx.y * TM;
  const int64_t q0 = (int64_t)blockIdx.x * TN;
  const int64_t boff = (int64_t)blockIdx.z * n * Q;
  const TI* inb = in + boff;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);

  for (int m0 = 0; m0 < n; m0 += TK) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int e = tid + 256 * r;
      const int pp = e >> 4, kk = e & 15;
      const int p = p0 + pp, mm = m0 + kk;
      Ms[kk][pp] = (p < n && mm < n) ? M[(int64_t)p * n + mm] : T(0);
      const int kk2 = e >> 6, qq = e & 63;
      const int mm2 = m0 + kk2;
      const int64_t q = q0 + qq;
      Is[kk2][qq] = (mm2 < n && q < Q) ? T(inb[(int64_t)mm2 * Q + q]) : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = Ms[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Is[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += a[r] * b[c];
    }
    __syncthreads();
  }
  TO* outb = out + boff;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + ty * 4 + r;
    if (p >= n) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t q = q0 + tx + 16 * c;
      if (q >= Q) continue;
      T v = acc[r][c];
      if (SCALE) {
        const int nx = tp.n[0];
        const int ia = (int)(q % nx), jb = (int)(q / nx);
        if (p == tp.null_index[2] && jb == tp.null_index[1] && ia == tp.null_index[0]) v = T(0);
        else v = v / (tp.lam[2][p] + tp.lam[1][jb] + tp.lam[0][ia]);
      }
      outb[(int64_t)p * Q + q] = TO(v);
    }
  }
}

// out[r][a] = sum_i in[r][i] M[a][i]   (rows R, n columns; x-axis transform)
template <typename T, typename TI, typename TO>
__global__ void __launch_bounds__(256) k_right(const T* __restrict__ M, const TI* __restrict__ in,
                                               TO* __restrict__ out, int n, int64_t R) {
  __shared__ T Is[TK][TM + 1];
  __shared__ T Ms[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = (int64_t)blockIdx.x * TM;
  const int a0 = blockIdx.y * TN;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = T(0);
  for (int i0 = 0; i0 < n; i0 += TK) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = tid + 256 * s;
      const int rr = e >> 4, kk = e & 15;
      const int64_t row = r0 + rr;
      const int ii = i0 + kk;
      Is[kk][rr] = (row < R && ii < n) ? T(in[row * n + ii]) : T(0);
      const int aa = rr;
      const int a = a0 + aa;
      Ms[kk][aa] = (a < n && ii < n) ? M[(int64_t)a * n + ii] : T(0);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      T x[4], y[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) x[r] = Is[kk][ty * 4 + r];
#pragma unroll
      for (int c = 0; c < 4; ++c) y[c] = Ms[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] += x[r] * y[c];
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t row = r0 + ty * 4 + r;
    if (row >= R) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = a0 + tx + 16 * c;
      if (a < n) out[row * n + a] = TO(acc[r][c]);
    }
  }
}

template <typename T, typename TI, typename TO>
fv_status run_right(const fv_grid* g, const T* M, const TI* in, TO* out) {
  const int n = g->n[0];
  const int64_t R = (int64_t)g->n[1] * g->n[2];
  dim3 grid((unsigned)((R + TM - 1) / TM), (n + TN - 1) / TN, 1);
  {
    LaunchScope ls_(g, FV_K_TPF_X);
    k_right<T, TI, TO><<<grid, 256, 0, g->stream>>>(M, in, out, n, R);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

template <typename T, typename TI, typename TO, bool SCALE>
fv_status run_left(const fv_grid* g, int axis, const T* M, const TI* in, TO* out,
                   const TpfDev<T>& tp) {
  const int n = g->n[axis];
  int64_t Q;
  int batch;
  if (axis == 1) { Q = g->n[0]; batch = g->n[2]; }
  else { Q = (int64_t)g->n[0] * g->n[1]; batch = 1; }
  dim3 grid((unsigned)((Q + TN - 1) / TN), (n + TM - 1) / TM, batch);
  {
    LaunchScope ls_(g, FV_K_TPF_YZ);
    k_left<T, TI, TO, SCALE><<<grid, 256, 0, g->stream>>>(M, in, out, n, Q, tp);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

template <typename T, typename TI, typename TO>
fv_status tpf_run(const fv_grid* g, const TpfDev<T>& tp, const TI* r, TO* phi) {
  T* a = (T*)g->tpf_buf[0];
  T* b = (T*)g->tpf_buf[1];
  FV_TRY((run_right<T, TI, T>(g, tp.Einv[0], r, a)));                  // x forward
  FV_TRY((run_left<T, T, T, false>(g, 1, tp.Einv[1], a, b, tp)));      // y forward
  FV_TRY((run_left<T, T, T, true>(g, 2, tp.Einv[2], b, a, tp)));       // z forward + scale
  FV_TRY((run_left<T, T, T, false>(g, 2, tp.E[2], a, b, tp)));         // z inverse
  FV_TRY((run_left<T, T, T, false>(g, 1, tp.E[1], b, a, tp)));         // y inverse
  FV_TRY((run_right<T, T, TO>(g, tp.E[0], a, phi)));                   // x inverse
  return FV_OK;
}

}  // namespace

fv_status tpf_solve(const fv_grid* g, const double* r, void* phi, int prec) {
  if (prec == FV_MIXED) return tpf_run<float, double, float>(g, g->tpf_f, r, (float*)phi);
  return tpf_run<double, double, double>(g, g->tpf_d, r, (double*)phi);
}

fv_status tpf_solve_f32(const fv_grid* g, const float* r, float* phi) {
  return tpf_run<float, float, float>(g, g->tpf_f, r, phi);
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_pressure_solve(const fv_grid* g, const double* r, double* phi, int prec) {
  if (!g || !r || !phi) { set_error("fv_pressure_solve: NULL argument"); return FV_EINVAL; }
  if (prec != FV_FP64 && prec != FV_MIXED) { set_error("fv_pressure_solve: bad prec"); return FV_EINVAL; }
  if (prec == FV_FP64) return tpf_solve(g, r, phi, FV_FP64);
  // mixed: float32 solve, widened into phi
  FV_TRY(launch_round_f32(g, r, g->r32, g->ncell));
  FV_TRY(tpf_solve_f32(g, g->r32, g->phi32));
  return launch_widen_f32(g, g->phi32, phi, g->ncell);
}

// ---------------------------------------------------------------------------
// Allocation-free pressure-correction solve.
//
// Some callers cannot allocate device memory: code that runs inside a
// memory pool it does not own, callers in the middle of a CUDA graph
// capture (where cudaMalloc is not allowed), or embedded users whose
// allocator is not reachable from this library.  For them
// fv_pressure_solve_noalloc runs the float32 tensor-product solve with all
// of its scratch (the per-axis eigenbases and the two transform buffers) in
// one file-scope device array of fixed size, so it calls no cudaMalloc,
// cudaFree or allocating library routine.  Limits: every dimension in
// [4, kNaMaxDim] and nx*ny*nz <= kNaMaxCells.  The array is shared by every
// call in the process: its contents are overwritten by each call (nothing in
// it needs to start at zero: the tables and both buffers are fully written
// before they are read), and calls that overlap on the GPU race on it.
namespace fv {
namespace {

constexpr int kNaMaxDim = 128;
constexpr int64_t kNaMaxCells = (int64_t)1 << 20;
constexpr int64_t kNaTables = 3 * (2 * (int64_t)kNaMaxDim * kNaMaxDim + kNaMaxDim);
constexpr int64_t kNaFloats = kNaTables + 2 * kNaMaxCells;

static __device__ __align__(256) float g_na_scratch[kNaFloats];

// device address of g_na_scratch per device, looked up once per device
static float* g_na_ptr[64] = {nullptr};

fv_status na_scratch_address(float** out) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_error("fv_pressure_solve_noalloc: device index out of range"); return FV_EINVAL; }
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    FV_CUDA(cudaGetSymbolAddress(&p, g_na_scratch));
    g_na_ptr[dev] = (float*)p;
  }
  *out = g_na_ptr[dev];
  return FV_OK;
}

template <typename TI, typename TO>
fv_status na_right(cudaStream_t st, int n, int64_t R, const float* M, const TI* in, TO* out) {
  dim3 grid((unsigned)((R + TM - 1) / TM), (n + TN - 1) / TN, 1);
  count_launch();
  k_right<float, TI, TO><<<grid, 256, 0, st>>>(M, in, out, n, R);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

template <bool SCALE>
fv_status na_left(cudaStream_t st, int n, int64_t Q, int batch, const float* M, const float* in,
                  float* out, const TpfDev<float>& tp) {
  dim3 grid((unsigned)((Q + TN - 1) / TN), (n + TM - 1) / TM, batch);
  count_launch();
  k_left<float, float, float, SCALE><<<grid, 256, 0, st>>>(M, in, out, n, Q, tp);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

}  // namespace

}  // namespace fv

extern "C" fv_status fv_pressure_solve_noalloc(int nx, int ny, int nz, int map, const double* r,
                                               double* phi, void* cuda_stream) {
  using namespace fv;
  if (!r || !phi) { set_error("fv_pressure_solve_noalloc: NULL pointer"); return FV_EINVAL; }
  if (map < 0 || map > 2) { set_error("fv_pressure_solve_noalloc: unknown map"); return FV_EINVAL; }
  const int n[3] = {nx, ny, nz};
  for (int d = 0; d < 3; ++d)
    if (n[d] < 4 || n[d] > kNaMaxDim) {
      set_error("fv_pressure_solve_noalloc: each dimension must be in [4, 128] (static scratch limit)");
      return FV_EINVAL;
    }
  const int64_t ncell = (int64_t)nx * ny * nz;
  if (ncell > kNaMaxCells) {
    set_error("fv_pressure_solve_noalloc: nx*ny*nz must be <= 1048576 (static scratch limit)");
    return FV_EINVAL;
  }
  float* base = nullptr;
  FV_TRY(na_scratch_address(&base));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // tables: E, Einv, lam per axis, packed at the start of the scratch array
  std::vector<float> tab;
  TpfDev<float> tp;
  size_t off[3][3];
  for (int d = 0; d < 3; ++d) {
    AxisBasis B;
    if (!host_axis_tables(n[d], map, B)) { set_error("fv_pressure_solve_noalloc: eigensolver failed"); return FV_ECUDA; }
    off[d][0] = tab.size();
    for (double v : B.E) tab.push_back((float)v);
    off[d][1] = tab.size();
    for (double v : B.Einv) tab.push_back((float)v);
    off[d][2] = tab.size();
    for (double v : B.lam) tab.push_back((float)v);
    tp.n[d] = n[d];
    tp.null_index[d] = B.null_index;
  }
  for (int d = 0; d < 3; ++d) {
    tp.E[d] = base + off[d][0];
    tp.Einv[d] = base + off[d][1];
    tp.lam[d] = base + off[d][2];
  }
  FV_CUDA(cudaMemcpyAsync(base, tab.data(), tab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  float* a = base + kNaTables;
  float* b = a + kNaMaxCells;
  const int64_t rows = (int64_t)ny * nz, qxy = (int64_t)nx * ny;
  FV_TRY((na_right<double, float>(st, nx, rows, tp.Einv[0], r, a)));   // x forward
  FV_TRY(na_left<false>(st, ny, nx, nz, tp.Einv[1], a, b, tp));       // y forward
  FV_TRY(na_left<true>(st, nz, qxy, 1, tp.Einv[2], b, a, tp));        // z forward + scale
  FV_TRY(na_left<false>(st, nz, qxy, 1, tp.E[2], a, b, tp));          // z inverse
  FV_TRY(na_left<false>(st, ny, nx, nz, tp.E[1], b, a, tp));          // y inverse
  FV_TRY((na_right<float, double>(st, nx, rows, tp.E[0], a, phi)));    // x inverse
  return FV_OK;
}
