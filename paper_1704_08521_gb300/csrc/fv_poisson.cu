// Pressure-correction solve of Section 3, step 1: D G phi = r with
// d phi/dn = 0, by tensor-product factorisation (the paper's TPF method).
// D G = L_x (+) L_y (+) L_z with L = E diag(lam) E^{-1} per axis, so
//   phi = (E_z (x) E_y (x) E_x) diag(1/(lam_x+lam_y+lam_z)) (E_z^-1 (x) E_y^-1 (x) E_x^-1) r
// with the single null mode (constant phi) set to zero.  Each 1-D transform
// is a dense contraction over one axis of the nz x ny x nx array, done by a
// register-tiled shared-memory kernel (64 x 64 outputs per block, 4 x 4 per
// thread); the eigenvalue scaling is fused into the epilogue of the third
// forward transform.  float32 in the mixed mode, float64 otherwise.
#include "fv_ff.cuh"
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


// float32 transform kernel of the mixed path: C(p,q) = sum_k A(p,k) B(k,q)
// for one batch entry b (blockIdx.z), with
//   A(p,k) = A[b*abs + p*lda + k]                (k contiguous)
//   B(k,q) = QN ? B[b*bbs + k*ldb + q]           (q contiguous)
//               : B[b*bbs + q*ldb + k]           (k contiguous)
//   C(p,q) = C[b*cbs + p*ldc + q]                (q contiguous)
// Block tile 64 (p) x 64 (q), K in chunks of 16 staged in shared memory;
// 256 threads with 4 x 4 outputs each (two float4 shared-memory reads per 16
// FMAs).  The next chunk is fetched into registers while the current one is
// multiplied, so the L2 latency of the operand loads overlaps the FMAs: at
// N = 100 a transform has only ~300 tiles (~2 per SM), too few warps to hide
// that latency by occupancy alone.  SCALE: the epilogue divides by
// lam_z[p] + lam_y[q / nx] + lam_x[q % nx] (null mode -> 0), the diagonal of
// the tensor-product solve.
constexpr int GP = 64, GQ = 64, GK = 16, GT = 256;

template <typename TA, typename TB, typename TO, bool QN, bool SCALE>
__global__ void __launch_bounds__(GT) k_gemm32(const TA* __restrict__ A, int64_t abs, int64_t lda,
                                               const TB* __restrict__ B, int64_t bbs, int64_t ldb,
                                               TO* __restrict__ C, int64_t cbs, int64_t ldc,
                                               int P, int64_t Q, int K, TpfDev<float> tp) {
  __shared__ __align__(16) float As[GK][GP + 4];
  __shared__ __align__(16) float Bs[GK][GQ + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int p0 = blockIdx.y * GP;
  const int64_t q0 = (int64_t)blockIdx.x * GQ;
  const TA* Ab = A + (int64_t)blockIdx.z * abs;
  const TB* Bb = B + (int64_t)blockIdx.z * bbs;
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
  float ra[4], rb[4];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = tid + GT * s;
      const int pp = e >> 4, kk = e & 15;
      const int p = p0 + pp, k = k0 + kk;
      ra[s] = (p < P && k < K) ? float(Ab[(int64_t)p * lda + k]) : 0.f;
      int kb, qq;
      if (QN) { kb = e >> 6; qq = e & 63; }
      else { kb = e & 15; qq = e >> 4; }
      const int k2 = k0 + kb;
      const int64_t q = q0 + qq;
      float v = 0.f;
      if (k2 < K && q < Q) v = QN ? float(Bb[(int64_t)k2 * ldb + q]) : float(Bb[q * ldb + k2]);
      rb[s] = v;
    }
  };
  auto stash = [&]() {
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const int e = tid + GT * s;
      As[e & 15][e >> 4] = ra[s];
      if (QN) Bs[e >> 6][e & 63] = rb[s];
      else Bs[e & 15][e >> 4] = rb[s];
    }
  };
  fetch(0);
  stash();
  __syncthreads();
  for (int k0 = 0; k0 < K; k0 += GK) {
    const bool more = k0 + GK < K;
    if (more) fetch(k0 + GK);
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
    if (more) {
      stash();
      __syncthreads();
    }
  }
  TO* Cb = C + (int64_t)blockIdx.z * cbs;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int p = p0 + ty * 4 + r;
    if (p >= P) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int64_t q = q0 + tx * 4 + c;
      if (q >= Q) continue;
      float v = acc[r][c];
      if (SCALE) {
        const int nx = tp.n[0];
        const int ia = (int)(q % nx), jb = (int)(q / nx);
        if (p == tp.null_index[2] && jb == tp.null_index[1] && ia == tp.null_index[0]) v = 0.f;
        else v = v / (tp.lam[2][p] + tp.lam[1][jb] + tp.lam[0][ia]);
      }
      if constexpr (sizeof(TO) == 8) Cb[(int64_t)p * ldc + q] = f32_to_f64(v);
      else Cb[(int64_t)p * ldc + q] = TO(v);
    }
  }
}

template <typename T, typename TI, typename TO>
fv_status run_right(const fv_grid* g, const T* M, const TI* in, TO* out) {
  if constexpr (sizeof(T) == 4) {
    // out[row][a] = sum_i in[row][i] M[a][i]: p = row, q = a, k = i
    const int n = g->n[0];
    const int64_t R = (int64_t)g->n[1] * g->n[2];
    dim3 grid((unsigned)((n + GQ - 1) / GQ), (unsigned)((R + GP - 1) / GP), 1);
    {
      LaunchScope ls_(g, FV_K_TPF_X);
      k_gemm32<TI, float, TO, false, false><<<grid, GT, 0, g->stream>>>(
          in, 0, n, M, 0, n, out, 0, n, (int)R, n, n, g->tpf_f);
    }
    FV_CHECK_LAUNCH();
    return FV_OK;
  }
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
  if constexpr (sizeof(T) == 4) {
    // out[b][p][q] = sum_m M[p][m] in[b][m][q]
    const int n = g->n[axis];
    int64_t Q;
    int batch;
    if (axis == 1) { Q = g->n[0]; batch = g->n[2]; }
    else { Q = (int64_t)g->n[0] * g->n[1]; batch = 1; }
    dim3 grid((unsigned)((Q + GQ - 1) / GQ), (unsigned)((n + GP - 1) / GP), batch);
    {
      LaunchScope ls_(g, FV_K_TPF_YZ);
      k_gemm32<float, TI, TO, true, SCALE><<<grid, GT, 0, g->stream>>>(
          M, 0, n, in, (int64_t)n * Q, Q, out, (int64_t)n * Q, Q, n, Q, n, g->tpf_f);
    }
    FV_CHECK_LAUNCH();
    return FV_OK;
  }
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


// ---------------------------------------------------------------------------
// Fused float32 tensor-product solve for grids with every dimension <= 128:
// three kernels instead of six transforms.
//   slab kernel (one block per z-plane k):  out_k = M2 (in_k M1^T)
//       forward: M1 = Ex^-1, M2 = Ey^-1;  inverse: M1 = Ex, M2 = Ey
//   column kernel (one block per 64 (x,y) columns):
//       out[:, q] = Ez diag(1 / (lam_x + lam_y + lam_z)) Ez^-1 in[:, q]
// Operands live in shared memory in k-major layout so that each thread's
// 4 x 4 outputs take one float4 read of each operand per k (8 FMA per
// shared load); the plane or column block is read from and written to
// global memory exactly once per kernel.
constexpr int kFusedMax = 128;
constexpr int kColGroup = 64;

__host__ __device__ __forceinline__ int up4(int n) { return (n + 3) & ~3; }
__host__ __device__ __forceinline__ int up8(int n) { return (n + 7) & ~7; }

// rows per thread of the fused kernels' register tiles (8 x 4 outputs:
// three float4 shared loads per 32 FMAs)
constexpr int RT = 8;

// acc[r][c] += sum_k At[k*lda + RT*tr + r] * Bt[k*ldb + 4*tc + c]
__device__ __forceinline__ void smem_mm(const float* At, int lda, const float* Bt, int ldb, int K,
                                        int tr, int tc, float (&acc)[RT][4]) {
#pragma unroll 2
  for (int k = 0; k < K; ++k) {
    const float4 a0 = *reinterpret_cast<const float4*>(At + k * lda + RT * tr);
    const float4 a1 = *reinterpret_cast<const float4*>(At + k * lda + RT * tr + 4);
    const float4 b = *reinterpret_cast<const float4*>(Bt + k * ldb + 4 * tc);
    const float av[RT] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
  }
}

// out[k][:, a0:a1] = M2 (in[k] M1[a0:a1, :]^T) for the (ny x nx) plane k and
// the column range of blockIdx.y (the plane's columns are split over
// gridDim.y blocks so that all SMs get work); M1t = M1^T (nx x nx), M2t =
// M2^T (ny x ny), both row-major.  Threads: (ceil(ny/4), ceil(ncol/4)).
__global__ void k_slab_xy(const float* __restrict__ in, float* __restrict__ out,
                          const float* __restrict__ M1t, const float* __restrict__ M2t, int nx,
                          int ny, int ncol) {
  extern __shared__ __align__(16) float sm[];
  const int a0 = blockIdx.y * ncol;
  const int na = min(ncol, nx - a0);
  const int ncp = up4(ncol), nyp = up8(ny);
  const int nmax = nx > ny ? nx : ny;
  float* A1 = sm;                      // in^T  [nx][nyp]; later M2t [ny][nyp]
  float* B1 = A1 + nmax * nyp;         // M1t[:, a0:a1]  [nx][ncp]
  float* T = B1 + nx * ncp;            // T     [nyp][ncp] (padded rows unused)
  const int nthr = blockDim.x;
  const int tid = threadIdx.x;
  const int tc = tid % (ncp / 4), tr = tid / (ncp / 4);
  const float* ink = in + (int64_t)blockIdx.x * nx * ny;
  {
    // (j, i) of element e = tid + s * nthr advanced without division
    const int dj = nthr / nx, di = nthr - dj * nx;
    int j = tid / nx, i = tid - j * nx;
#pragma unroll 4
    for (int e = tid; e < nx * ny; e += nthr) {
      A1[i * nyp + j] = ink[e];
      i += di;
      j += dj;
      if (i >= nx) { i -= nx; ++j; }
    }
  }
  {
    const int dr = nthr / ncol, dc = nthr - dr * ncol;
    int r = tid / ncol, c = tid - r * ncol;
#pragma unroll 4
    for (int e = tid; e < nx * ncol; e += nthr) {
      B1[r * ncp + c] = (c < na) ? M1t[r * nx + a0 + c] : 0.f;
      c += dc;
      r += dr;
      if (c >= ncol) { c -= ncol; ++r; }
    }
  }
  __syncthreads();
  float acc[RT][4] = {};
  smem_mm(A1, nyp, B1, ncp, nx, tr, tc, acc);       // T[j][a] = sum_i in[j][i] M1[a][i]
#pragma unroll
  for (int r = 0; r < RT; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) T[(RT * tr + r) * ncp + 4 * tc + c] = acc[r][c];
  __syncthreads();
  {
    const int dj = nthr / ny, db = nthr - dj * ny;
    int j = tid / ny, b = tid - j * ny;
#pragma unroll 4
    for (int e = tid; e < ny * ny; e += nthr) {
      A1[j * nyp + b] = M2t[e];
      b += db;
      j += dj;
      if (b >= ny) { b -= ny; ++j; }
    }
  }
  __syncthreads();
  float acc2[RT][4] = {};
  smem_mm(A1, nyp, T, ncp, ny, tr, tc, acc2);       // out[b][a] = sum_j M2[b][j] T[j][a]
  float* outk = out + (int64_t)blockIdx.x * nx * ny;
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int b = RT * tr + r;
    if (b >= ny) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int a = 4 * tc + c;
      if (a < na) outk[b * nx + a0 + a] = acc2[r][c];
    }
  }
}

// z-direction forward transform, eigenvalue scaling and inverse transform for
// 64 (x,y) columns.  Threads: (ceil(nz/4), 16).
__global__ void k_col_z(const float* __restrict__ in, float* __restrict__ out, TpfDev<float> tp) {
  extern __shared__ __align__(16) float sm[];
  const int nx = tp.n[0], ny = tp.n[1], nz = tp.n[2];
  const int nzp = up8(nz);
  const int64_t Q = (int64_t)nx * ny;
  const int64_t q0 = (int64_t)blockIdx.x * kColGroup;
  float* X = sm;                        // in tile   [nz][64]
  float* Mz = X + nz * kColGroup;       // Ez^-T / Ez^T [nz][nzp]
  float* Tt = Mz + nz * nzp;            // scaled     [nzp][64]
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int tc = tid & 15, tr = tid >> 4;
#pragma unroll 8
  for (int e = tid; e < nz * kColGroup; e += nthr) {
    const int k = e >> 6, qq = e & 63;   // power-of-two split: shifts only
    const int64_t q = q0 + qq;
    X[e] = (q < Q) ? in[(int64_t)k * Q + q] : 0.f;
  }
  const float* Zi = tp.Einvt[2];
  {
    const int dk = nthr / nz, dc = nthr - dk * nz;
    int k = tid / nz, c = tid - k * nz;
#pragma unroll 4
    for (int e = tid; e < nz * nz; e += nthr) {
      Mz[k * nzp + c] = Zi[e];
      c += dc;
      k += dk;
      if (c >= nz) { c -= nz; ++k; }
    }
  }
  __syncthreads();
  float acc[RT][4] = {};
  smem_mm(Mz, nzp, X, kColGroup, nz, tr, tc, acc);   // t[c][q] = sum_k Ez^-1[c][k] in[k][q]
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int c = RT * tr + r;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int64_t q = q0 + 4 * tc + cc;
      float v = 0.f;
      if (c < nz && q < Q) {
        const int ia = (int)(q % nx), jb = (int)(q / nx);
        if (!(c == tp.null_index[2] && jb == tp.null_index[1] && ia == tp.null_index[0]))
          v = acc[r][cc] / (tp.lam[2][c] + tp.lam[1][jb] + tp.lam[0][ia]);
      }
      Tt[c * kColGroup + 4 * tc + cc] = v;
    }
  }
  __syncthreads();
  const float* Ze = tp.Et[2];
  {
    const int dc = nthr / nz, dm = nthr - dc * nz;
    int c = tid / nz, m = tid - c * nz;
#pragma unroll 4
    for (int e = tid; e < nz * nz; e += nthr) {
      Mz[c * nzp + m] = Ze[e];
      m += dm;
      c += dc;
      if (m >= nz) { m -= nz; ++c; }
    }
  }
  __syncthreads();
  float acc2[RT][4] = {};
  smem_mm(Mz, nzp, Tt, kColGroup, nz, tr, tc, acc2);  // out[m][q] = sum_c Ez[m][c] t[c][q]
#pragma unroll
  for (int r = 0; r < RT; ++r) {
    const int m = RT * tr + r;
    if (m >= nz) continue;
#pragma unroll
    for (int cc = 0; cc < 4; ++cc) {
      const int64_t q = q0 + 4 * tc + cc;
      if (q < Q) out[(int64_t)m * Q + q] = acc2[r][cc];
    }
  }
}

// the columns of a plane are split over kSlabSplit blocks
constexpr int kSlabSplit = 1;
inline int slab_cols(int nx) { return (nx + kSlabSplit - 1) / kSlabSplit; }

inline size_t slab_smem(int nx, int ny) {
  const int nmax = nx > ny ? nx : ny;
  const int ncp = up4(slab_cols(nx));
  return sizeof(float) * ((size_t)nmax * up8(ny) + (size_t)nx * ncp + (size_t)up8(ny) * ncp);
}

inline size_t col_smem(int nz) {
  return sizeof(float) * ((size_t)nz * kColGroup + (size_t)nz * up8(nz) + (size_t)up8(nz) * kColGroup);
}

fv_status tpf_fused_f32(const fv_grid* g, const float* r, float* phi) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const TpfDev<float>& tp = g->tpf_f;
  float* a = (float*)g->tpf_buf[0];
  float* b = (float*)g->tpf_buf[1];
  const size_t ss = slab_smem(nx, ny), cs = col_smem(nz);
  static bool attr_set = false;   // the attribute is per function, not per grid
  if (!attr_set) {
    FV_CUDA(cudaFuncSetAttribute(k_slab_xy, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    FV_CUDA(cudaFuncSetAttribute(k_col_z, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr_set = true;
  }
  const int slab_threads = (up8(ny) / RT) * (up4(slab_cols(nx)) / 4);
  const dim3 slab_grid(nz, kSlabSplit);
  const int col_threads = (up8(nz) / RT) * 16;
  const unsigned ncol = (unsigned)(((int64_t)nx * ny + kColGroup - 1) / kColGroup);
  {
    LaunchScope ls_(g, FV_K_TPF_X);
    k_slab_xy<<<slab_grid, slab_threads, ss, g->stream>>>(r, a, tp.Einvt[0], tp.Einvt[1], nx, ny,
                                                          slab_cols(nx));
  }
  FV_CHECK_LAUNCH();
  {
    LaunchScope ls_(g, FV_K_TPF_YZ);
    k_col_z<<<ncol, col_threads, cs, g->stream>>>(a, b, tp);
  }
  FV_CHECK_LAUNCH();
  {
    LaunchScope ls_(g, FV_K_TPF_X);
    k_slab_xy<<<slab_grid, slab_threads, ss, g->stream>>>(b, phi, tp.Et[0], tp.Et[1], nx, ny,
                                                          slab_cols(nx));
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

inline bool fused_ok(const fv_grid* g) {
  return g->n[0] <= kFusedMax && g->n[1] <= kFusedMax && g->n[2] <= kFusedMax &&
         slab_smem(g->n[0], g->n[1]) <= 200 * 1024 && col_smem(g->n[2]) <= 200 * 1024;
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
  if (fused_ok(g)) return tpf_fused_f32(g, r, phi);
  return tpf_run<float, float, float>(g, g->tpf_f, r, phi);
}

// one float32 transform along `axis` (0: x, 1: y, 2: z) between the two
// transform buffers, for kernel timing
fv_status tpf_one_transform_f32(const fv_grid* g, int axis) {
  float* a = (float*)g->tpf_buf[0];
  float* b = (float*)g->tpf_buf[1];
  if (fused_ok(g)) {          // fused kernels: axis 0 = one slab kernel, else one column kernel
    const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
    if (axis == 0) {
      LaunchScope ls_(g, FV_K_TPF_X);
      k_slab_xy<<<dim3(nz, kSlabSplit), (up8(ny) / RT) * (up4(slab_cols(nx)) / 4),
                  slab_smem(nx, ny), g->stream>>>(a, b, g->tpf_f.Einvt[0], g->tpf_f.Einvt[1], nx,
                                                  ny, slab_cols(nx));
    } else {
      LaunchScope ls_(g, FV_K_TPF_YZ);
      k_col_z<<<(unsigned)(((int64_t)nx * ny + kColGroup - 1) / kColGroup), (up8(nz) / RT) * 16,
                col_smem(nz), g->stream>>>(a, b, g->tpf_f);
    }
    FV_CHECK_LAUNCH();
    return FV_OK;
  }
  if (axis == 0) return run_right<float, float, float>(g, g->tpf_f.Einv[0], a, b);
  return run_left<float, float, float, false>(g, axis, g->tpf_f.Einv[axis], a, b, g->tpf_f);
}

}  // namespace fv

using namespace fv;

extern "C" fv_status fv_pressure_solve(const fv_grid* g, const double* r, double* phi, int prec) {
  if (!g || !r || !phi) { set_error("fv_pressure_solve: NULL argument"); return FV_EINVAL; }
  if (prec != FV_FP64 && prec != FV_MIXED && prec != FV_FF) { set_error("fv_pressure_solve: bad prec"); return FV_EINVAL; }
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
