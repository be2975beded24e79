// Pressure-correction solve of Section 3, step 1: D G phi = r with
// d phi/dn = 0, by tensor-product factorisation (the paper's TPF method).
// D G = L_x (+) L_y (+) L_z with L = E diag(lam) E^{-1} per axis, so
//   phi = (E_z (x) E_y (x) E_x) diag(1/(lam_x+lam_y+lam_z)) (E_z^-1 (x) E_y^-1 (x) E_x^-1) r
// with the single null mode (constant phi) set to zero.  Each 1-D transform
// is a dense contraction over one axis of the nz x ny x nx array, done by a
// register-tiled shared-memory kernel (64 x 64 outputs per block, 4 x 4 per
// thread); the eigenvalue scaling is fused into the epilogue of the third
// forward transform.  float32 in the mixed mode, float64 otherwise.
#include <atomic>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <vector>

#include "fv_ff.cuh"
#include "fv_internal.cuh"
#include "fv_tc5.cuh"

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
          M, 0, n, in, (int64_t)n * Q, Q, out, (int64_t)n * Q, Q, n, Q, n, tp);
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

// The fused kernels run the dense contractions on the 5th-generation tensor
// cores (tcgen05.mma kind::tf32, accumulators in tensor memory) with every
// operand split into TF32 hi + lo parts and three products per product,
//   a b ~ a_lo b_hi + a_hi b_lo + a_hi b_hi   (a_lo b_lo is below float32
// round-off), which keeps the transforms at float32-level accuracy (~22
// significant bits).  One block owns a 128-row accumulator (rows padded to
// 128); one thread issues the MMAs and commits them to an mbarrier that the
// block waits on (with an iteration limit: on timeout the block sets the
// grid's sticky fault word, which the SIMPLE loop reports as FV_ETIMEOUT, and
// its outputs become NaN).  The eigenbases come pre-split and
// pre-laid-out (TcMats) and are copied to shared memory with 16-byte
// cp.async; field values are split by the threads that store them.

__device__ __forceinline__ uint32_t tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

constexpr int kMbarLimit = 1 << 22;   // polls of an mbarrier before the block gives up

__host__ __device__ __forceinline__ int up16(int n) { return (n + 15) & ~15; }

inline uint32_t tmem_cols(int n) {
  uint32_t c = 32;
  while ((int)c < n) c <<= 1;
  return c;
}

// copy [hi | lo] (2 * count floats, contiguous) into two shared arrays
__device__ __forceinline__ void stage_pair(const float* __restrict__ src, float* hi, float* lo, int count,
                                           int tid, int nthr) {
  const int half = count >> 2;   // float4 per half
  for (int e = tid; e < 2 * half; e += nthr)
    tc5::cp_async16(e < half ? hi + 4 * e : lo + 4 * (e - half), src + 4 * e);
}

// issue D (+)= A B^T over K (multiple of 8) as three split products per step
__device__ __forceinline__ void issue_split_gemm(uint32_t tmem, const float* Ah, const float* Al,
                                                 const float* Bh, const float* Bl, int K, int N) {
  const uint32_t idesc = tc5::idesc_tf32(128, N);
  const uint32_t sbo = (uint32_t)(K / 4) * 128;
  const uint32_t ah = tc5::smem_u32(Ah), al = tc5::smem_u32(Al), bh = tc5::smem_u32(Bh),
                 bl = tc5::smem_u32(Bl);
  for (int ks = 0; ks < K / 8; ++ks) {
    const uint32_t off = (uint32_t)ks * 256;   // 8 elements of K: two 16-byte core-matrix columns
    tc5::mma_tf32(tmem, tc5::sdesc(al + off, 128, sbo), tc5::sdesc(bh + off, 128, sbo), idesc, ks > 0);
    tc5::mma_tf32(tmem, tc5::sdesc(ah + off, 128, sbo), tc5::sdesc(bl + off, 128, sbo), idesc, 1);
    tc5::mma_tf32(tmem, tc5::sdesc(ah + off, 128, sbo), tc5::sdesc(bh + off, 128, sbo), idesc, 1);
  }
}

// asynchronous 4-byte global -> shared copy; zero-fills when !valid (src unread)
__device__ __forceinline__ void cp_async4(float* dst, const float* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(tc5::smem_u32(dst)), "l"(src),
               "r"(valid ? 4 : 0)
               : "memory");
}

constexpr int kUmmaThreads = 256;   // 8 warps: warps w and w + 4 share accumulator lanes 32 (w % 4) ..

__device__ __forceinline__ float4 split4(float4& v) {   // v -> lo parts, returns hi parts
  float4 h;
  h.x = __uint_as_float(tf32_rna(v.x)); v.x = __uint_as_float(tf32_rna(v.x - h.x));
  h.y = __uint_as_float(tf32_rna(v.y)); v.y = __uint_as_float(tf32_rna(v.y - h.y));
  h.z = __uint_as_float(tf32_rna(v.z)); v.z = __uint_as_float(tf32_rna(v.z - h.z));
  h.w = __uint_as_float(tf32_rna(v.w)); v.w = __uint_as_float(tf32_rna(v.w - h.w));
  return h;
}

// Both 1-D transforms of the (ny x nx) plane k = blockIdx.x for the columns
// [a0, a0 + Na) of chunk blockIdx.y (Na a multiple of 16, <= 128):
//   GEMM 1 (transposed):  T^T[a][j] = sum_i M1[a0 + a][i] in[k][j][i]
//                         M = 128 (a), N = N1 = up16(ny) (j), K = up8(nx) (i)
//   GEMM 2:               out[k][b][a0 + a] = sum_j M2[b][j] T^T[a][j]
//                         M = 128 (b), N = Na (a), K = up8(ny) (j)
// The plane is copied with cp.async straight into its canonical positions
// (16-byte runs of 4 columns; vec: nx % 4 == 0 so that every full run is
// 16-byte aligned in global memory) and split in place by the thread that
// copied it.  256 threads; warps w and w + 4 own accumulator rows
// 32 (w % 4) .. + 31, the first and second half of the columns.
__global__ void __launch_bounds__(kUmmaThreads) k_slab_umma(const float* __restrict__ in,
                                                            float* __restrict__ out,
                                                            const float* __restrict__ bx,
                                                            const float* __restrict__ ay, int nx, int ny,
                                                            int Na, uint32_t tcols, int vec,
                                                            unsigned* __restrict__ fault) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int K1 = up8(nx), K2 = up8(ny), Km = K1 > K2 ? K1 : K2;
  const int N1 = up16(ny), Nb = N1 > Na ? N1 : Na;
  float* Ah = reinterpret_cast<float*>(sm);
  float* Al = Ah + 128 * Km;
  float* Bh = Al + 128 * Km;
  float* Bl = Bh + Nb * Km;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = blockIdx.x, a0 = blockIdx.y * Na;
  tc5::pdl_trigger();
  if (warp == 0) tc5::tmem_alloc(&tslot, tcols);
  if (tid == 0) tc5::mbar_init(&bar, 1);
  // M1 chunk [hi | lo] (128 x K1) -> region A
  stage_pair(bx + (size_t)blockIdx.y * 2 * 128 * K1, Ah, Al, 128 * K1, tid, kUmmaThreads);
  // everything above uses constants only; the field is the predecessor's output
  tc5::pdl_wait();
  // the plane (N1 x K1: rows j, columns i) -> Bl in canonical order; a warp
  // pass covers 8 rows x 4 runs (lane: row 8 rb + lane % 8, run 4 kq + lane / 8)
  const float* ink = in + (size_t)k * nx * ny;
  const int kb4 = K1 >> 2, kq4 = (kb4 + 3) >> 2;
  const int sbo1 = kb4 * 32;   // floats per 8-row block
  for (int t = warp; t < (N1 >> 3) * kq4; t += 8) {
    const int rb = t / kq4, kq = t - rb * kq4;
    const int j = 8 * rb + (lane & 7), kb = 4 * kq + (lane >> 3);
    if (kb < kb4) {
      float* dst = Bl + rb * sbo1 + kb * 32 + (lane & 7) * 4;
      const int i0 = 4 * kb;
      if (vec && j < ny && i0 + 3 < nx) {
        tc5::cp_async16(dst, ink + j * nx + i0);
      } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const bool ok = j < ny && i0 + q < nx;
          cp_async4(dst + q, ok ? ink + j * nx + i0 + q : ink, ok);
        }
      }
    }
  }
  tc5::cp_async_wait_all();
  for (int t = warp; t < (N1 >> 3) * kq4; t += 8) {
    const int rb = t / kq4, kq = t - rb * kq4;
    const int kb = 4 * kq + (lane >> 3);
    if (kb < kb4) {
      const int o = rb * sbo1 + kb * 32 + (lane & 7) * 4;
      float4 v = *reinterpret_cast<float4*>(Bl + o);
      const float4 h = split4(v);
      *reinterpret_cast<float4*>(Bh + o) = h;
      *reinterpret_cast<float4*>(Bl + o) = v;
    }
  }
  tc5::fence_proxy_async();
  tc5::fence_before_sync();
  __syncthreads();
  tc5::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    issue_split_gemm(tmem, Ah, Al, Bh, Bl, K1, N1);
    tc5::commit(&bar);
  }
  const bool ok1 = tc5::mbar_wait(&bar, 0, kMbarLimit);
  __syncwarp();   // tcgen05.ld is warp-collective
  tc5::fence_after_sync();
  // region A is free: stage M2 while T^T moves from tensor memory to region B
  stage_pair(ay, Ah, Al, 128 * K2, tid, kUmmaThreads);
  const int row = 32 * (warp & 3) + lane;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  {
    const int half = ((N1 >> 3) + 1) >> 1;   // 8-column chunks of the first half
    const int c_begin = warp < 4 ? 0 : 8 * half, c_end = warp < 4 ? 8 * half : N1;
    for (int c = c_begin; c < c_end; c += 8) {
      float v[8];
      tc5::ld8(trow + (uint32_t)c, v);
      if (row < Na && c < K2) {
        float4 lo0 = make_float4(v[0], v[1], v[2], v[3]), lo1 = make_float4(v[4], v[5], v[6], v[7]);
        if (!ok1) lo0 = lo1 = make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
        const float4 hi0 = split4(lo0), hi1 = split4(lo1);
        const uint32_t o = tc5::canon_offset(row, c, K2) >> 2;
        *reinterpret_cast<float4*>(Bh + o) = hi0;
        *reinterpret_cast<float4*>(Bh + o + 32) = hi1;
        *reinterpret_cast<float4*>(Bl + o) = lo0;
        *reinterpret_cast<float4*>(Bl + o + 32) = lo1;
      }
    }
  }
  tc5::cp_async_wait_all();
  tc5::fence_proxy_async();
  tc5::fence_before_sync();
  __syncthreads();
  tc5::fence_after_sync();
  if (tid == 0) {
    issue_split_gemm(tmem, Ah, Al, Bh, Bl, K2, Na);
    tc5::commit(&bar);
  }
  const bool ok2 = tc5::mbar_wait(&bar, 1, kMbarLimit);
  __syncwarp();
  tc5::fence_after_sync();
  if (tid == 0 && !(ok1 && ok2)) atomicOr(fault, 1u);   // reported as FV_ETIMEOUT
  {
    float* outr = out + (size_t)k * nx * ny + (size_t)row * nx;
    const int half = ((Na >> 3) + 1) >> 1;
    const int c_begin = warp < 4 ? 0 : 8 * half, c_end = warp < 4 ? 8 * half : Na;
    for (int c = c_begin; c < c_end; c += 8) {
      float v[8];
      tc5::ld8(trow + (uint32_t)c, v);
      if (!ok2) v[0] = __int_as_float(0x7fc00000);
      const int a = a0 + c;
      if (row < ny) {
        if (vec && a + 7 < nx) {
          *reinterpret_cast<float4*>(outr + a) = make_float4(v[0], v[1], v[2], v[3]);
          *reinterpret_cast<float4*>(outr + a + 4) = make_float4(v[4], v[5], v[6], v[7]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            if (a + q < nx) outr[a + q] = v[q];
        }
      }
    }
  }
  tc5::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tmem, tcols);
}

// z transform, eigenvalue scaling and inverse z transform of the N (x, y)
// columns q0 + [0, N), q = j nx + i:
//   t[c][q] = sum_k Ez^-1[c][k] in[k][q] / (lam_z[c] + lam_y[j] + lam_x[i])  (null mode -> 0)
//   out[m][q] = sum_c Ez[m][c] t[c][q]
// GEMM 1: A = Ez^-1, B = in^T; GEMM 2: A = Ez, B = t^T.  256 threads (as above).
// The input tile is copied in its own order (16-byte runs along q) into a
// padded row-major tile R and transposed + split from there into the
// canonical operand; the scaled intermediate goes through a per-warp 32 x 9
// transpose scratch (in R) so that both land as 16-byte runs.
// vec: Q % 4 == 0 and N % 4 == 0 (16-byte aligned global runs).
__global__ void __launch_bounds__(kUmmaThreads) k_col_umma(const float* __restrict__ in,
                                                           float* __restrict__ out, TpfDev<float> tp,
                                                           const float* __restrict__ azi,
                                                           const float* __restrict__ aze, int N,
                                                           uint32_t tcols, int vec,
                                                           unsigned* __restrict__ fault) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tslot;
  const int nx = tp.n[0], ny = tp.n[1], nz = tp.n[2];
  const int Kz = up8(nz);
  const int64_t Q = (int64_t)nx * ny, q0 = (int64_t)blockIdx.x * N;
  float* Ah = reinterpret_cast<float*>(sm);
  float* Al = Ah + 128 * Kz;
  float* Bh = Al + 128 * Kz;
  float* Bl = Bh + N * Kz;
  float* lamq = Bl + N * Kz;
  int* nullq = reinterpret_cast<int*>(lamq + N);
  const int ldR = N + 4;
  float* R = reinterpret_cast<float*>(nullq + N);   // Kz x ldR raw tile, later transpose scratch
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  tc5::pdl_trigger();
  if (warp == 0) tc5::tmem_alloc(&tslot, tcols);
  if (tid == 0) tc5::mbar_init(&bar, 1);
  stage_pair(azi, Ah, Al, 128 * Kz, tid, kUmmaThreads);
  // everything above uses constants only; the field is the predecessor's output
  tc5::pdl_wait();
  // the tile in[kk][q0 .. q0 + N) -> R in 16-byte runs (rows kk >= nz and
  // columns beyond Q zero-filled)
  {
    const int n4 = N >> 2;
    for (int e = tid; e < Kz * n4; e += kUmmaThreads) {
      const int kk = e / n4, j4 = e - kk * n4;
      float* dst = R + kk * ldR + 4 * j4;
      const int64_t qq = q0 + 4 * j4;
      if (vec && kk < nz && qq + 3 < Q) {
        tc5::cp_async16(dst, in + kk * Q + qq);
      } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const bool ok = kk < nz && qq + i < Q;
          cp_async4(dst + i, ok ? in + kk * Q + qq + i : in, ok);
        }
      }
    }
  }
  for (int q = tid; q < N; q += kUmmaThreads) {
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
  tc5::cp_async_wait_all();
  __syncthreads();
  // transpose + split: run (q, kb) = R[4 kb .. 4 kb + 3][q] -> canonical (q, 4 kb);
  // a warp covers 8 consecutive q x 4 consecutive kb (512 contiguous bytes)
  {
    const int kb4 = Kz >> 2;
    for (int e = tid; e < N * kb4; e += kUmmaThreads) {
      const int ql = e & 7, rest = e >> 3;
      const int qh = rest / kb4, kb = rest - qh * kb4;
      const int q = 8 * qh + ql;
      const float* rp = R + 4 * kb * ldR + q;
      float4 v = make_float4(rp[0], rp[ldR], rp[2 * ldR], rp[3 * ldR]);
      const float4 h = split4(v);
      const uint32_t o = tc5::canon_offset(q, 4 * kb, Kz) >> 2;
      *reinterpret_cast<float4*>(Bh + o) = h;
      *reinterpret_cast<float4*>(Bl + o) = v;
    }
  }
  tc5::fence_proxy_async();
  tc5::fence_before_sync();
  __syncthreads();
  tc5::fence_after_sync();
  const uint32_t tmem = tslot;
  if (tid == 0) {
    issue_split_gemm(tmem, Ah, Al, Bh, Bl, Kz, N);
    tc5::commit(&bar);
  }
  const bool ok1 = tc5::mbar_wait(&bar, 0, kMbarLimit);
  __syncwarp();   // tcgen05.ld is warp-collective
  tc5::fence_after_sync();
  stage_pair(aze, Ah, Al, 128 * Kz, tid, kUmmaThreads);
  const int row = 32 * (warp & 3) + lane;   // c of GEMM 1, m of GEMM 2
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  const int half = ((N >> 3) + 1) >> 1;
  const int c_begin = warp < 4 ? 0 : 8 * half, c_end = warp < 4 ? 8 * half : N;
  {
    const float lz = row < nz ? tp.lam[2][row] : 1.f;
    const bool nullrow = row == tp.null_index[2];
    float* scr = R + warp * (32 * 9);   // this warp's 32 x 8 block, row pitch 9
    const int ql = lane & 7, rg = lane >> 3;
    for (int c = c_begin; c < c_end; c += 8) {
      float v[8];
      tc5::ld8(trow + (uint32_t)c, v);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int col = c + q;
        float t = 0.f;
        if (row < nz && q0 + col < Q && !(nullrow && nullq[col])) t = v[q] / (lz + lamq[col]);
        if (!ok1) t = __int_as_float(0x7fc00000);
        scr[lane * 9 + q] = t;
      }
      __syncwarp();
      // lane: column c + ql, rows 4 rg .. 4 rg + 3 and 4 (rg + 4) .. + 3 of the warp's 32
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int r0 = 4 * (rg + 4 * hh);
        const int grow = 32 * (warp & 3) + r0;
        if (grow < Kz) {
          float4 t4 = make_float4(scr[r0 * 9 + ql], scr[(r0 + 1) * 9 + ql], scr[(r0 + 2) * 9 + ql],
                                  scr[(r0 + 3) * 9 + ql]);
          const float4 h4 = split4(t4);
          const uint32_t o = tc5::canon_offset(c + ql, grow, Kz) >> 2;
          *reinterpret_cast<float4*>(Bh + o) = h4;
          *reinterpret_cast<float4*>(Bl + o) = t4;
        }
      }
      __syncwarp();
    }
  }
  tc5::cp_async_wait_all();
  tc5::fence_proxy_async();
  tc5::fence_before_sync();
  __syncthreads();
  tc5::fence_after_sync();
  if (tid == 0) {
    issue_split_gemm(tmem, Ah, Al, Bh, Bl, Kz, N);
    tc5::commit(&bar);
  }
  const bool ok2 = tc5::mbar_wait(&bar, 1, kMbarLimit);
  __syncwarp();
  tc5::fence_after_sync();
  if (tid == 0 && !(ok1 && ok2)) atomicOr(fault, 1u);   // reported as FV_ETIMEOUT
  for (int c = c_begin; c < c_end; c += 8) {
    float v[8];
    tc5::ld8(trow + (uint32_t)c, v);
    if (!ok2) v[0] = __int_as_float(0x7fc00000);
    if (row < nz) {
      float* o = out + row * Q + q0 + c;
      if (vec && q0 + c + 7 < Q) {
        *reinterpret_cast<float4*>(o) = make_float4(v[0], v[1], v[2], v[3]);
        *reinterpret_cast<float4*>(o + 4) = make_float4(v[4], v[5], v[6], v[7]);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q)
          if (q0 + c + q < Q) o[q] = v[q];
      }
    }
  }
  tc5::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc5::tmem_dealloc(tmem, tcols);
}

inline size_t slab_smem(int nx, int ny, int Na) {
  const int Km = up8(nx) > up8(ny) ? up8(nx) : up8(ny);
  const int Nb = up16(ny) > Na ? up16(ny) : Na;
  return sizeof(float) * (size_t)(2 * 128 + 2 * Nb) * Km;
}

inline size_t col_smem(int nz, int N) {
  // eigenbasis hi / lo, operand hi / lo, lam / null per column, raw tile R (>= 8 x 32 x 9 scratch)
  const size_t R = (size_t)up8(nz) * (N + 4) > 8 * 32 * 9 ? (size_t)up8(nz) * (N + 4) : 8 * 32 * 9;
  return sizeof(float) * ((size_t)(2 * 128 + 2 * N) * up8(nz) + 2 * (size_t)N + R);
}

constexpr size_t kSmemCap = 220 * 1024;

// launch shapes, fixed per grid: the slab kernel covers a plane's columns in
// one chunk (up16(nx) <= 128); the column kernel takes N columns per block so
// that its blocks cover the SMs once (N a multiple of 16, <= 128)
inline void tc_shapes(int nx, int ny, int nz, int* nsplit, int* slab_n, int* col_n) {
  *nsplit = 1;
  *slab_n = up16(nx);
  const int64_t Q = (int64_t)nx * ny;
  int n = up16((int)((Q + 151) / 152));
  if (n > 128) n = 128;
  while (n > 16 && col_smem(nz, n) > kSmemCap) n -= 16;
  *col_n = n;
}

fv_status set_tc_attributes() {
  static bool done = false;   // the attribute is per function, not per grid
  if (!done) {
    FV_CUDA(cudaFuncSetAttribute(k_slab_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    FV_CUDA(cudaFuncSetAttribute(k_col_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap));
    done = true;
  }
  return FV_OK;
}

// Launch with programmatic stream serialization: the kernel's constant
// set-up (tensor-memory allocation, eigenbasis staging) overlaps the tail of
// the kernel before it; its pdl_wait() orders every use of that kernel's
// output.  Captured into the evaluation graphs as a programmatic edge.
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// dir 0: forward (Einv) transforms, 1: inverse (E)
fv_status launch_slab(const fv_grid* g, const float* in, float* out, int dir) {
  // dir 0: forward x-y transforms, dir 1: inverse
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int N = g->tc.slab_n;
  LaunchScope ls_(g, dir == 0 ? FV_K_TPF_X : FV_K_TPF_XINV);
  FV_CUDA(launch_pdl(k_slab_umma, dim3(nz, g->tc.slab_nsplit), dim3(kUmmaThreads),
                     slab_smem(nx, ny, N), g->stream, in, out, (const float*)g->tc.bx[dir],
                     (const float*)g->tc.ay[dir], nx, ny, N,
                     tmem_cols(up16(ny) > N ? up16(ny) : N),
                     (nx % 4 == 0 && N % 4 == 0) ? 1 : 0, g->d_fault));
  return FV_OK;
}

fv_status launch_col(const fv_grid* g, const float* in, float* out) {
  const int N = g->tc.col_n;
  const int64_t Q = (int64_t)g->n[0] * g->n[1];
  LaunchScope ls_(g, FV_K_TPF_YZ);
  FV_CUDA(launch_pdl(k_col_umma, dim3((unsigned)((Q + N - 1) / N)), dim3(kUmmaThreads),
                     col_smem(g->n[2], N), g->stream, in, out, g->tpf_f,
                     (const float*)g->tc.az[0], (const float*)g->tc.az[1], N, tmem_cols(N),
                     (Q % 4 == 0 && N % 4 == 0) ? 1 : 0, g->d_fault));
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

// [hi | lo] of the rows x kdim operand whose element (r, k) is f(r, k), in
// the canonical K-major layout
template <typename F>
static void lay_out(int rows, int kdim, F f, float* out) {
  const size_t half = (size_t)rows * kdim;
  for (int r = 0; r < rows; ++r)
    for (int k = 0; k < kdim; ++k) {
      const double x = f(r, k);
      const float hi = tf32_host((float)x);
      const float lo = tf32_host((float)(x - (double)hi));
      const size_t o = tc5::canon_offset(r, k, kdim) / 4;
      out[o] = hi;
      out[half + o] = lo;
    }
}

fv_status build_tc_mats(fv_grid* g) {
  g->tc = TcMats();
  for (int d = 0; d < 3; ++d)
    if (g->n[d] > kFusedMax) return FV_OK;   // the fused kernels serve n <= 128 at most
  const int nx = g->n[0], ny = g->n[1], nz = g->n[2];
  const int K1 = up8(nx), K2 = up8(ny), Kz = up8(nz);
  int ns, N, Nc;
  tc_shapes(nx, ny, nz, &ns, &N, &Nc);
  // the plane operand (up16(ny) x up8(nx)) and the eigenbasis (128 rows) must
  // fit one block's shared memory together (n up to about 112); larger grids
  // take the unfused transforms
  if (slab_smem(nx, ny, N) > kSmemCap || col_smem(nz, Nc) > kSmemCap) return FV_OK;
  const size_t szb = (size_t)ns * 2 * 128 * K1, sza = (size_t)2 * 128 * K2, szz = (size_t)2 * 128 * Kz;
  const size_t total = 2 * szb + 2 * sza + 2 * szz;
  std::vector<float> h(total, 0.f);
  float* p = h.data();
  size_t off_bx[2], off_ay[2], off_az[2], o = 0;
  for (int dir = 0; dir < 2; ++dir) { off_bx[dir] = o; o += szb; }
  for (int dir = 0; dir < 2; ++dir) { off_ay[dir] = o; o += sza; }
  for (int q = 0; q < 2; ++q) { off_az[q] = o; o += szz; }
  for (int dir = 0; dir < 2; ++dir) {
    const std::vector<double>& Mx = dir == 0 ? g->basis[0].Einv : g->basis[0].E;
    const std::vector<double>& My = dir == 0 ? g->basis[1].Einv : g->basis[1].E;
    const std::vector<double>& Mz = dir == 0 ? g->basis[2].Einv : g->basis[2].E;
    for (int c = 0; c < ns; ++c) {
      const int a0 = c * N;
      lay_out(128, K1,
              [&](int r, int k) { return (r < N && a0 + r < nx && k < nx) ? Mx[(size_t)(a0 + r) * nx + k] : 0.0; },
              p + off_bx[dir] + (size_t)c * 2 * 128 * K1);
    }
    lay_out(128, K2, [&](int r, int k) { return (r < ny && k < ny) ? My[(size_t)r * ny + k] : 0.0; },
            p + off_ay[dir]);
    lay_out(128, Kz, [&](int r, int k) { return (r < nz && k < nz) ? Mz[(size_t)r * nz + k] : 0.0; },
            p + off_az[dir]);
  }
  cudaError_t e = cudaMalloc(&g->d_tc, total * sizeof(float));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    g->d_tc = nullptr;
    set_error("cudaMalloc of the tensor-core operands failed");
    return FV_ENOMEM;
  }
  g->ws_bytes += (int64_t)(total * sizeof(float));
  FV_CUDA(cudaMemcpy(g->d_tc, h.data(), total * sizeof(float), cudaMemcpyHostToDevice));
  const float* base = (const float*)g->d_tc;
  for (int q = 0; q < 2; ++q) {
    g->tc.bx[q] = base + off_bx[q];
    g->tc.ay[q] = base + off_ay[q];
    g->tc.az[q] = base + off_az[q];
  }
  g->tc.slab_nsplit = ns;
  g->tc.slab_n = N;
  g->tc.col_n = Nc;
  g->tc.ready = true;
  return FV_OK;
}

// One float64 1-D transform out = M applied along `axis` (0 x, 1 y, 2 z) of
// the nz x ny x nx array `in` (the unfused kernels of the pressure solve)
fv_status transform_axis_f64(const fv_grid* g, int axis, const double* M, const double* in,
                             double* out) {
  if (axis == 0) return run_right<double, double, double>(g, M, in, out);
  return run_left<double, double, double, false>(g, axis, M, in, out, g->tpf_d);
}

// The unfused float32 tensor-product solve with the tables of tp (the
// pressure operator's, or those of another separable operator)
fv_status tpf_run_f32(const fv_grid* g, const TpfDev<float>& tp, const float* r, float* phi) {
  return tpf_run<float, float, float>(g, tp, r, phi);
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
    return axis == 2 ? launch_col(g, a, b) : launch_slab(g, a, b, axis);
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
// memory pool it does not own and may not grow, or embedded users whose
// allocator is not reachable from this library.  For them
// fv_pressure_solve_noalloc runs the float32 tensor-product solve with all
// of its scratch (the per-axis eigenbases and the two transform buffers) in
// one file-scope device array of fixed size, so it calls no cudaMalloc,
// cudaFree or allocating library routine.  Limits: every dimension in
// [4, kNaMaxDim] and nx*ny*nz <= kNaMaxCells.  The array is shared by every
// call in the process: its contents are overwritten by each call (nothing in
// it needs to start at zero: the tables and both buffers are fully written
// before they are read), and calls that overlap on the GPU race on it.
//
// The module that holds the array is loaded lazily (CUDA's default), so the
// first call on a device, which looks up the array's device address with
// cudaGetSymbolAddress, is the one that makes the driver reserve the array;
// later calls reserve nothing.
//
// The host-side eigenbasis tables of an axis (n, map) are computed once and
// kept for the life of the process (an immutable cache under a mutex), so
// the asynchronous upload of a call always reads memory that outlives it and
// later calls do not repeat the O(n^3) eigensolve.
namespace fv {
namespace {

constexpr int kNaMaxDim = 128;
constexpr int64_t kNaMaxCells = (int64_t)1 << 20;
constexpr int64_t kNaTables = 3 * (2 * (int64_t)kNaMaxDim * kNaMaxDim + kNaMaxDim);
constexpr int64_t kNaFloats = kNaTables + 2 * kNaMaxCells;

static __device__ __align__(256) float g_na_scratch[kNaFloats];

// device address of g_na_scratch per device, looked up once per device
static std::atomic<float*> g_na_ptr[64];

fv_status na_scratch_address(float** out) {
  int dev = 0;
  FV_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) { set_error("fv_pressure_solve_noalloc: device index out of range"); return FV_EINVAL; }
  float* p = g_na_ptr[dev].load(std::memory_order_acquire);
  if (!p) {
    // two threads that race here both store the same address
    void* q = nullptr;
    FV_CUDA(cudaGetSymbolAddress(&q, g_na_scratch));
    p = (float*)q;
    g_na_ptr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return FV_OK;
}

// float32 [E | Einv | lam] of one axis, built once per (n, map)
struct NaAxis {
  std::vector<float> tab;
  int null_index = 0;
};

const NaAxis* na_axis_tables(int n, int map) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, std::unique_ptr<NaAxis>> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find({n, map});
  if (it != cache.end()) return it->second.get();
  AxisBasis B;
  if (!host_axis_tables(n, map, B)) return nullptr;
  auto a = std::make_unique<NaAxis>();
  a->tab.reserve(2 * (size_t)n * n + n);
  for (double v : B.E) a->tab.push_back((float)v);
  for (double v : B.Einv) a->tab.push_back((float)v);
  for (double v : B.lam) a->tab.push_back((float)v);
  a->null_index = B.null_index;
  const NaAxis* r = a.get();
  cache.emplace(std::make_pair(n, map), std::move(a));
  return r;
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
  TpfDev<float> tp;
  float* dst = base;
  for (int d = 0; d < 3; ++d) {
    const NaAxis* A = na_axis_tables(n[d], map);
    if (!A) { set_error("fv_pressure_solve_noalloc: eigensolver failed"); return FV_ECUDA; }
    const size_t nn = (size_t)n[d] * n[d];
    tp.n[d] = n[d];
    tp.null_index[d] = A->null_index;
    tp.E[d] = dst;
    tp.Einv[d] = dst + nn;
    tp.lam[d] = dst + 2 * nn;
    FV_CUDA(cudaMemcpyAsync(dst, A->tab.data(), A->tab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
    dst += A->tab.size();
  }
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
