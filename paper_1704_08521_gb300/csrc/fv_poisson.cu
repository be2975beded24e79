// Pressure-correction solve of Section 3, step 1: D G phi = r with
// d phi/dn = 0, by tensor-product factorisation (the paper's TPF method).
// D G = L_x (+) L_y (+) L_z with L = E diag(lam) E^{-1} per axis, so
//   phi = (E_z (x) E_y (x) E_x) diag(1/(lam_x+lam_y+lam_z)) (E_z^-1 (x) E_y^-1 (x) E_x^-1) r
// with the single null mode (constant phi) set to zero.  Each 1-D transform
// is a dense contraction over one axis of the nz x ny x nx array, done by a
// register-tiled shared-memory kernel (64 x 64 outputs per block, 4 x 4 per
// thread); the eigenvalue scaling is fused into the epilogue of the third
// forward transform.  float32 in the mixed mode, float64 otherwise.
#include <cstring>
#include <vector>

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

__host__ __device__ __forceinline__ int up8(int n) { return (n + 7) & ~7; }

// The fused kernels run the dense contractions on the tensor cores
// (mma.sync m16n8k8, TF32 operands, float32 accumulation) with every operand
// split into TF32 hi + lo parts and three products per tile,
//   a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi   (the a_lo b_lo term is below
// float32 round-off), which keeps the transforms at float32-level accuracy
// (~22 significant bits) while using the tensor pipes instead of the FP32
// lanes.  The eigenbases come pre-split in fragment order (TcFrags); field
// values are split when staged in shared memory or when loaded into a
// fragment.

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_rna(x);
  lo = tf32_rna(x - __uint_as_float(hi));   // exact difference, rounded to TF32
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t f2u(float x) { return __float_as_uint(x); }

// asynchronous 4-byte global -> shared copy; zero-fills when !valid (src unread)
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(valid ? 4 : 0)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

constexpr int kTcMaxNt = 8;   // n-tiles (8 columns each) per block of the slab kernel
constexpr int kTcCols = 32;   // (x, y) columns per block of the column kernel

__host__ __device__ __forceinline__ int up16(int n) { return (n + 15) & ~15; }

// smallest leading dimension >= n (multiple of 8) that is 8 or 24 mod 32:
// the B-fragment reads (rows t4, columns g) then hit 32 distinct banks
inline int ld_b(int n) {
  int ld = up8(n);
  while (ld % 32 != 8 && ld % 32 != 24) ld += 8;
  return ld;
}

// Both 1-D transforms of one (ny x nx) plane k = blockIdx.x, restricted to
// the columns [a0, a0 + ncol) of blockIdx.y:
//   T[j][a] = sum_i in[k][j][i] M1[a][i]     (x, tensor cores, B = bx frags)
//   out[k][b][a] = sum_j M2[b][j] T[j][a]    (y, tensor cores, A = ay frags)
// One warp per 16-row tile (blockDim = 32 * up16(ny) / 16).  Shared memory:
// P [16 MT][ldP] (the plane, zero-padded), T hi / lo [16 MT][ldT].
__global__ void __launch_bounds__(256) k_slab_xy_tc(const float* __restrict__ in,
                                                    float* __restrict__ out,
                                                    const float4* __restrict__ bx,
                                                    const float4* __restrict__ ay, int nx, int ny,
                                                    int ncol, int ldP, int ldT) {
  extern __shared__ __align__(16) float sm[];
  const int MT = blockDim.x >> 5;
  const int KS1 = up8(nx) >> 3, KS2 = up8(ny) >> 3;
  float* P = sm;
  float* Th = P + 16 * MT * ldP;
  float* Tl = Th + 16 * MT * ldT;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t4 = lane & 3;
  const int a0 = blockIdx.y * ncol;
  const int nt0 = a0 >> 3;
  const int ntc = min(ncol >> 3, KS1 - nt0);
  const int kp = up8(nx);
  const float* ink = in + (int64_t)blockIdx.x * nx * ny;
  for (int j = warp; j < 16 * MT; j += MT)
    for (int i = lane; i < kp; i += 32) {
      const bool ok = j < ny && i < nx;
      cp_async4(P + j * ldP + i, ok ? ink + j * nx + i : ink, ok);
    }
  cp_async_wait_all();
  __syncthreads();

  float acc[kTcMaxNt][4];
#pragma unroll
  for (int n = 0; n < kTcMaxNt; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float* Pw = P + (16 * warp + g) * ldP + t4;
  const float4* bw = bx + (size_t)nt0 * KS1 * 32 + lane;   // [n][ks] stride KS1 * 32
  float4 bcur[kTcMaxNt], bnxt[kTcMaxNt];
#pragma unroll
  for (int n = 0; n < kTcMaxNt; ++n)
    if (n < ntc) bcur[n] = __ldg(bw + (size_t)n * KS1 * 32);
  for (int ks = 0; ks < KS1; ++ks) {
    if (ks + 1 < KS1) {
#pragma unroll
      for (int n = 0; n < kTcMaxNt; ++n)
        if (n < ntc) bnxt[n] = __ldg(bw + (size_t)n * KS1 * 32 + (ks + 1) * 32);
    }
    uint32_t ah[4], al[4];
    split_tf32(Pw[8 * ks], ah[0], al[0]);
    split_tf32(Pw[8 * ks + 8 * ldP], ah[1], al[1]);
    split_tf32(Pw[8 * ks + 4], ah[2], al[2]);
    split_tf32(Pw[8 * ks + 8 * ldP + 4], ah[3], al[3]);
    // the three products sweep the n-tiles in turn: consecutive mma on one
    // accumulator are ntc instructions apart
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) mma_tf32(acc[n], al, f2u(bcur[n].x), f2u(bcur[n].y));
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) mma_tf32(acc[n], ah, f2u(bcur[n].z), f2u(bcur[n].w));
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) {
        mma_tf32(acc[n], ah, f2u(bcur[n].x), f2u(bcur[n].y));
        bcur[n] = bnxt[n];
      }
  }
  {
    const int r0 = 16 * warp + g;
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n) {
      if (n < ntc) {
        const int c = 8 * n + 2 * t4;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int o = (r0 + 8 * (q >> 1)) * ldT + c + (q & 1);
          uint32_t h, l;
          split_tf32(acc[n][q], h, l);
          Th[o] = __uint_as_float(h);
          Tl[o] = __uint_as_float(l);
        }
      }
    }
  }
  __syncthreads();

#pragma unroll
  for (int n = 0; n < kTcMaxNt; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float4* aw = ay + (size_t)warp * KS2 * 64 + 2 * lane;
  float4 h4n = __ldg(aw), l4n = __ldg(aw + 1);
  for (int ks = 0; ks < KS2; ++ks) {
    const float4 h4 = h4n, l4 = l4n;
    if (ks + 1 < KS2) {
      h4n = __ldg(aw + (ks + 1) * 64);
      l4n = __ldg(aw + (ks + 1) * 64 + 1);
    }
    const uint32_t ah[4] = {f2u(h4.x), f2u(h4.y), f2u(h4.z), f2u(h4.w)};
    const uint32_t al[4] = {f2u(l4.x), f2u(l4.y), f2u(l4.z), f2u(l4.w)};
    const int o = (8 * ks + t4) * ldT + g;
    uint32_t bh[kTcMaxNt][2], bl[kTcMaxNt][2];
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) {
        const int on = o + 8 * n;
        bh[n][0] = f2u(Th[on]);
        bh[n][1] = f2u(Th[on + 4 * ldT]);
        bl[n][0] = f2u(Tl[on]);
        bl[n][1] = f2u(Tl[on + 4 * ldT]);
      }
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) mma_tf32(acc[n], al, bh[n][0], bh[n][1]);
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) mma_tf32(acc[n], ah, bl[n][0], bl[n][1]);
#pragma unroll
    for (int n = 0; n < kTcMaxNt; ++n)
      if (n < ntc) mma_tf32(acc[n], ah, bh[n][0], bh[n][1]);
  }
  float* outk = out + (int64_t)blockIdx.x * nx * ny;
  const int b0 = 16 * warp + g;
#pragma unroll
  for (int n = 0; n < kTcMaxNt; ++n) {
    if (n < ntc) {
      const int a = a0 + 8 * n + 2 * t4;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int b = b0 + 8 * (q >> 1), aa = a + (q & 1);
        if (b < ny && aa < nx) outk[b * nx + aa] = acc[n][q];
      }
    }
  }
}

// z-direction forward transform, eigenvalue scaling and inverse transform of
// kTcCols (x, y) columns q0 + [0, kTcCols), q = j nx + i:
//   t[c][q] = sum_k Ez^-1[c][k] in[k][q] / (lam_z[c] + lam_y[j] + lam_x[i])   (null mode -> 0)
//   out[m][q] = sum_c Ez[m][c] t[c][q]
// One warp per 16-row tile (blockDim = 32 * up16(nz) / 16).  Shared memory:
// X hi / lo [16 MT][ldX] (input, then t), lam_x + lam_y and the null flag per column.
__global__ void __launch_bounds__(256) k_col_z_tc(const float* __restrict__ in,
                                                  float* __restrict__ out, TpfDev<float> tp,
                                                  const float4* __restrict__ azi,
                                                  const float4* __restrict__ aze, int ldX) {
  extern __shared__ __align__(16) float sm[];
  const int nx = tp.n[0], ny = tp.n[1], nz = tp.n[2];
  const int MT = blockDim.x >> 5, KS = up8(nz) >> 3;
  const int64_t Q = (int64_t)nx * ny;
  const int64_t q0 = (int64_t)blockIdx.x * kTcCols;
  float* Xh = sm;
  float* Xl = Xh + 16 * MT * ldX;
  float* lamq = Xl + 16 * MT * ldX;
  int* nullq = reinterpret_cast<int*>(lamq + kTcCols);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  for (int k = warp; k < 16 * MT; k += MT)
    for (int q = lane; q < kTcCols; q += 32) {
      const bool ok = k < nz && q0 + q < Q;
      cp_async4(Xh + k * ldX + q, ok ? in + k * Q + q0 + q : in, ok);
    }
  for (int q = tid; q < kTcCols; q += blockDim.x) {
    const int64_t qq = q0 + q;
    float lq = 1.f;
    int nl = 0;
    if (qq < Q) {
      const int ia = (int)(qq % nx), jb = (int)(qq / nx);
      lq = tp.lam[0][ia] + tp.lam[1][jb];
      nl = (ia == tp.null_index[0] && jb == tp.null_index[1]);
    }
    lamq[q] = lq;
    nullq[q] = nl;
  }
  cp_async_wait_all();
  // each thread splits the elements it copied (same indices as the copy loop)
  for (int k = warp; k < 16 * MT; k += MT)
    for (int q = lane; q < kTcCols; q += 32) {
      uint32_t h, l;
      split_tf32(Xh[k * ldX + q], h, l);
      Xh[k * ldX + q] = __uint_as_float(h);
      Xl[k * ldX + q] = __uint_as_float(l);
    }
  __syncthreads();

  constexpr int NT = kTcCols / 8;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  const float4* aw = azi + (size_t)warp * KS * 64 + 2 * lane;
  float4 h4n = __ldg(aw), l4n = __ldg(aw + 1);
  for (int ks = 0; ks < KS; ++ks) {
    const float4 h4 = h4n, l4 = l4n;
    if (ks + 1 < KS) {
      h4n = __ldg(aw + (ks + 1) * 64);
      l4n = __ldg(aw + (ks + 1) * 64 + 1);
    }
    const uint32_t ah[4] = {f2u(h4.x), f2u(h4.y), f2u(h4.z), f2u(h4.w)};
    const uint32_t al[4] = {f2u(l4.x), f2u(l4.y), f2u(l4.z), f2u(l4.w)};
    const int o = (8 * ks + t4) * ldX + g;
    uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int on = o + 8 * n;
      bh[n][0] = f2u(Xh[on]);
      bh[n][1] = f2u(Xh[on + 4 * ldX]);
      bl[n][0] = f2u(Xl[on]);
      bl[n][1] = f2u(Xl[on + 4 * ldX]);
    }
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], al, bh[n][0], bh[n][1]);
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], ah, bl[n][0], bl[n][1]);
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], ah, bh[n][0], bh[n][1]);
  }
  __syncthreads();   // every warp is done reading X: t overwrites it
  {
    const int c0 = 16 * warp + g;
#pragma unroll
    for (int n = 0; n < NT; ++n) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = c0 + 8 * (q >> 1), col = 8 * n + 2 * t4 + (q & 1);
        float v = 0.f;
        if (c < nz && q0 + col < Q && !(c == tp.null_index[2] && nullq[col]))
          v = acc[n][q] / (tp.lam[2][c] + lamq[col]);
        uint32_t h, l;
        split_tf32(v, h, l);
        Xh[c * ldX + col] = __uint_as_float(h);
        Xl[c * ldX + col] = __uint_as_float(l);
      }
    }
  }
  __syncthreads();

#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n][0] = acc[n][1] = acc[n][2] = acc[n][3] = 0.f;
  aw = aze + (size_t)warp * KS * 64 + 2 * lane;
  h4n = __ldg(aw);
  l4n = __ldg(aw + 1);
  for (int ks = 0; ks < KS; ++ks) {
    const float4 h4 = h4n, l4 = l4n;
    if (ks + 1 < KS) {
      h4n = __ldg(aw + (ks + 1) * 64);
      l4n = __ldg(aw + (ks + 1) * 64 + 1);
    }
    const uint32_t ah[4] = {f2u(h4.x), f2u(h4.y), f2u(h4.z), f2u(h4.w)};
    const uint32_t al[4] = {f2u(l4.x), f2u(l4.y), f2u(l4.z), f2u(l4.w)};
    const int o = (8 * ks + t4) * ldX + g;
    uint32_t bh[NT][2], bl[NT][2];
#pragma unroll
    for (int n = 0; n < NT; ++n) {
      const int on = o + 8 * n;
      bh[n][0] = f2u(Xh[on]);
      bh[n][1] = f2u(Xh[on + 4 * ldX]);
      bl[n][0] = f2u(Xl[on]);
      bl[n][1] = f2u(Xl[on + 4 * ldX]);
    }
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], al, bh[n][0], bh[n][1]);
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], ah, bl[n][0], bl[n][1]);
#pragma unroll
    for (int n = 0; n < NT; ++n) mma_tf32(acc[n], ah, bh[n][0], bh[n][1]);
  }
  const int m0 = 16 * warp + g;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + 8 * (q >> 1);
      const int64_t col = q0 + 8 * n + 2 * t4 + (q & 1);
      if (m < nz && col < Q) out[m * Q + col] = acc[n][q];
    }
  }
}

// launch shapes of the fused kernels
struct SlabShape {
  int nsplit, ncol, ldP, ldT, threads;
  size_t smem;
};

inline SlabShape slab_shape(int nx, int ny, int nz) {
  SlabShape s;
  const int kp = up8(nx);
  // column split: at least enough for 8 n-tiles per block; among up to 4,
  // the one whose nz * nsplit blocks fill whole waves of 2 blocks per SM best
  const int nmin = (kp + 8 * kTcMaxNt - 1) / (8 * kTcMaxNt);
  s.nsplit = nmin;
  double best = -1.0;
  for (int ns = nmin; ns <= 4 && 8 * ns <= kp; ++ns) {
    const int64_t blocks = (int64_t)nz * ns, slots = 2 * 152;
    const double eff = (double)blocks / (double)(((blocks + slots - 1) / slots) * slots);
    if (eff > best + 1e-9) { best = eff; s.nsplit = ns; }
  }
  s.ncol = up8((kp + s.nsplit - 1) / s.nsplit);
  s.ldP = kp + 4;                 // ldP / 4 odd: the A-fragment reads hit 32 banks
  s.ldT = ld_b(s.ncol);
  s.threads = 32 * (up16(ny) / 16);
  s.smem = sizeof(float) * (size_t)up16(ny) * (s.ldP + 2 * s.ldT);
  return s;
}

struct ColShape {
  int ldX, threads;
  unsigned blocks;
  size_t smem;
};

inline ColShape col_shape(int nx, int ny, int nz) {
  ColShape c;
  c.ldX = ld_b(kTcCols);
  c.threads = 32 * (up16(nz) / 16);
  c.blocks = (unsigned)(((int64_t)nx * ny + kTcCols - 1) / kTcCols);
  c.smem = sizeof(float) * ((size_t)2 * up16(nz) * c.ldX + 2 * kTcCols);
  return c;
}

fv_status set_tc_attributes() {
  static bool done = false;   // the attribute is per function, not per grid
  if (!done) {
    FV_CUDA(cudaFuncSetAttribute(k_slab_xy_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    FV_CUDA(cudaFuncSetAttribute(k_col_z_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    done = true;
  }
  return FV_OK;
}

// dir 0: forward (Einv) transforms, 1: inverse (E)
fv_status launch_slab(const fv_grid* g, const float* in, float* out, int dir) {
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const SlabShape s = slab_shape(nx, ny, nz);
  LaunchScope ls_(g, FV_K_TPF_X);
  k_slab_xy_tc<<<dim3(nz, s.nsplit), s.threads, s.smem, g->stream>>>(
      in, out, g->tc.bx[dir], g->tc.ay[dir], nx, ny, s.ncol, s.ldP, s.ldT);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status launch_col(const fv_grid* g, const float* in, float* out) {
  const ColShape c = col_shape(g->n[0], g->n[1], g->n[2]);
  LaunchScope ls_(g, FV_K_TPF_YZ);
  k_col_z_tc<<<c.blocks, c.threads, c.smem, g->stream>>>(in, out, g->tpf_f, g->tc.az[0], g->tc.az[1],
                                                         c.ldX);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status tpf_fused_f32(const fv_grid* g, const float* r, float* phi) {
  FV_TRY(set_tc_attributes());
  float* a = (float*)g->tpf_buf[0];
  float* b = (float*)g->tpf_buf[1];
  FV_TRY(launch_slab(g, r, a, 0));
  FV_TRY(launch_col(g, a, b));
  FV_TRY(launch_slab(g, b, phi, 1));
  return FV_OK;
}

inline bool fused_ok(const fv_grid* g) {
  return g->tc.ready && g->n[0] <= kFusedMax && g->n[1] <= kFusedMax && g->n[2] <= kFusedMax;
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

// TF32 value of x, rounded to nearest with ties away from zero (cvt.rna)
static float tf32_host(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x1000u) & 0xffffe000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

static void split_host(double x, float& hi, float& lo) {
  hi = tf32_host((float)x);
  lo = tf32_host((float)(x - (double)hi));
}

// B fragments of M (n x n, row-major): B[k = i][col = a] = M[a][i]
static void frag_b(const std::vector<double>& M, int n, float4* out) {
  const int KS = up8(n) / 8;
  for (int nt = 0; nt < KS; ++nt)
    for (int ks = 0; ks < KS; ++ks)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t4 = lane & 3;
        const int a = 8 * nt + g, i0 = 8 * ks + t4, i1 = i0 + 4;
        const double v0 = (a < n && i0 < n) ? M[(size_t)a * n + i0] : 0.0;
        const double v1 = (a < n && i1 < n) ? M[(size_t)a * n + i1] : 0.0;
        float h0, l0, h1, l1;
        split_host(v0, h0, l0);
        split_host(v1, h1, l1);
        out[((size_t)nt * KS + ks) * 32 + lane] = make_float4(h0, h1, l0, l1);
      }
}

// A fragments of M (n x n, row-major): A[row = r][k = c] = M[r][c]
static void frag_a(const std::vector<double>& M, int n, float4* out) {
  const int KS = up8(n) / 8, MT = up16(n) / 16;
  for (int mt = 0; mt < MT; ++mt)
    for (int ks = 0; ks < KS; ++ks)
      for (int lane = 0; lane < 32; ++lane) {
        const int g = lane >> 2, t4 = lane & 3;
        const int r[4] = {16 * mt + g, 16 * mt + g + 8, 16 * mt + g, 16 * mt + g + 8};
        const int c[4] = {8 * ks + t4, 8 * ks + t4, 8 * ks + t4 + 4, 8 * ks + t4 + 4};
        float h[4], l[4];
        for (int q = 0; q < 4; ++q)
          split_host((r[q] < n && c[q] < n) ? M[(size_t)r[q] * n + c[q]] : 0.0, h[q], l[q]);
        float4* o = out + (((size_t)mt * KS + ks) * 32 + lane) * 2;
        o[0] = make_float4(h[0], h[1], h[2], h[3]);
        o[1] = make_float4(l[0], l[1], l[2], l[3]);
      }
}

fv_status build_tc_frags(fv_grid* g) {
  g->tc = TcFrags();
  for (int d = 0; d < 3; ++d)
    if (g->n[d] > kFusedMax) return FV_OK;   // the fused kernels serve n <= 128 only
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const size_t szb = (size_t)(up8(nx) / 8) * (up8(nx) / 8) * 32;
  const size_t sza_y = (size_t)(up16(ny) / 16) * (up8(ny) / 8) * 64;
  const size_t sza_z = (size_t)(up16(nz) / 16) * (up8(nz) / 8) * 64;
  const size_t total = 2 * (szb + sza_y + sza_z);
  std::vector<float4> h(total);
  float4* p = h.data();
  float4* bx[2] = {p, p + szb};
  float4* ay[2] = {p + 2 * szb, p + 2 * szb + sza_y};
  float4* az[2] = {p + 2 * szb + 2 * sza_y, p + 2 * szb + 2 * sza_y + sza_z};
  frag_b(g->basis[0].Einv, nx, bx[0]);
  frag_b(g->basis[0].E, nx, bx[1]);
  frag_a(g->basis[1].Einv, ny, ay[0]);
  frag_a(g->basis[1].E, ny, ay[1]);
  frag_a(g->basis[2].Einv, nz, az[0]);
  frag_a(g->basis[2].E, nz, az[1]);
  cudaError_t e = cudaMalloc(&g->d_tc, total * sizeof(float4));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    g->d_tc = nullptr;
    set_error("cudaMalloc of the tensor-core fragments failed");
    return FV_ENOMEM;
  }
  g->ws_bytes += (int64_t)(total * sizeof(float4));
  FV_CUDA(cudaMemcpy(g->d_tc, h.data(), total * sizeof(float4), cudaMemcpyHostToDevice));
  const float4* base = (const float4*)g->d_tc;
  for (int q = 0; q < 2; ++q) {
    g->tc.bx[q] = base + (bx[q] - p);
    g->tc.ay[q] = base + (ay[q] - p);
    g->tc.az[q] = base + (az[q] - p);
  }
  g->tc.ready = true;
  return FV_OK;
}

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
    FV_TRY(set_tc_attributes());
    return axis == 0 ? launch_slab(g, a, b, 0) : launch_col(g, a, b);
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
