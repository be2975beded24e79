// Learned initial guess of the pressure correction (no counterpart in the
// paper; an optional first pass of the SIMPLE-like loop of Section 3).
//
// A 3-D convolutional U-Net of 4 levels (16/32/48/64 channels, two 3x3x3
// convolutions + ReLU per level, 2x2x2 mean pooling, nearest upsampling,
// skip concatenation, a 1x1x1 float32 output layer) maps the float32
// right-hand side r = D w of the pressure equation plus three metric
// channels (log of the local cell widths) to a guess of phi.  Weights and
// activations are BF16, every contraction accumulates in float32.
//
// Kernels:
//   k_conv3   3x3x3 convolution, zero padding, as an implicit GEMM on the
//             BF16 tensor cores (mma.sync m16n8k16): rows = cells (16 per
//             warp), columns = output channels, reduction = 27 taps x input
//             channels; bias + ReLU fused into the epilogue.  The same kernel
//             computes the data gradient with flipped, channel-transposed
//             weights.
//   k_wgrad   weight gradient per tap, dW_tap = dY^T X_tap, also on the BF16
//             tensor cores; cells split over blocks, float32 atomics.
//   the rest  pooling, upsampling, ReLU masks, output layer, the mean-free
//             mean-square loss and Adam are element-wise kernels.
// Layout: activations channel-last ([cell][channel], cells x fastest), every
// channel count a multiple of 16 (the 4 input channels are zero-padded to 16).
// Parameters (float32 master copy, BF16 mirror): per convolution c the
// weights W_c[27][cout][cin] (tap t = 9 (dz+1) + 3 (dy+1) + (dx+1)) then the
// bias b_c[cout]; finally the output layer's 16 weights and 1 bias.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "fv_internal.cuh"

namespace fv {
namespace unet {

typedef __nv_bfloat16 bf16;

struct Dims {
  int nx, ny, nz;
};

// convolution layers: (level, cin, cout); level 0 is the finest
struct ConvSpec {
  int level, cin, cout;
};
constexpr int kNConv = 14;
constexpr ConvSpec kConvs[kNConv] = {
    {0, 16, 16},  {0, 16, 16},    // encoder level 0
    {1, 16, 32},  {1, 32, 32},    // encoder level 1
    {2, 32, 48},  {2, 48, 48},    // encoder level 2
    {3, 48, 64},  {3, 64, 64},    // bottom
    {2, 112, 48}, {2, 48, 48},    // decoder level 2: up(64) ++ skip(48)
    {1, 80, 32},  {1, 32, 32},    // decoder level 1: up(48) ++ skip(32)
    {0, 48, 16},  {0, 16, 16},    // decoder level 0: up(32) ++ skip(16)
};

__device__ __forceinline__ uint32_t pack2(bf16 lo, bf16 hi) {
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// cell index of the neighbour of (i, j, k) at tap t, or -1 outside the box
__device__ __forceinline__ int neighbour(const Dims& d, int i, int j, int k, int t) {
  const int a = i + t % 3 - 1, b = j + (t / 3) % 3 - 1, c = k + t / 9 - 1;
  if (a < 0 || a >= d.nx || b < 0 || b >= d.ny || c < 0 || c >= d.nz) return -1;
  return (c * d.ny + b) * d.nx + a;
}

// Y[cell][co] = act(bias[co] + sum_{t, ci} X[nb(cell, t)][ci] W[t][co][ci]).
// X has row stride cin (multiple of 16), Y row stride COUT.  One warp
// computes 16 cells x COUT channels; rows past the last cell are masked.
template <int COUT, bool RELU>
__global__ void __launch_bounds__(128) k_conv3(const bf16* __restrict__ X, int cin,
                                               const bf16* __restrict__ W,
                                               const float* __restrict__ bias,
                                               bf16* __restrict__ Y, Dims d) {
  const int ncell = d.nx * d.ny * d.nz;
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t4 = lane & 3;
  const int c0 = warp * 16;
  if (c0 >= ncell) return;
  int row[2], ci[2], cj[2], ck[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = c0 + g + 8 * h;
    row[h] = c < ncell ? c : -1;
    const int cc = c < ncell ? c : 0;
    ci[h] = cc % d.nx;
    cj[h] = (cc / d.nx) % d.ny;
    ck[h] = cc / (d.nx * d.ny);
  }
  constexpr int NT = COUT / 8;
  float acc[NT][4];
#pragma unroll
  for (int n = 0; n < NT; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
  const uint32_t* X32 = reinterpret_cast<const uint32_t*>(X);
  const uint32_t* W32 = reinterpret_cast<const uint32_t*>(W);
  for (int t = 0; t < 27; ++t) {
    int nb[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) nb[h] = row[h] >= 0 ? neighbour(d, ci[h], cj[h], ck[h], t) : -1;
    for (int k0 = 0; k0 < cin; k0 += 16) {
      // A fragment (16 cells x 16 channels): rows g / g+8, columns 2t4.. / 2t4+8..
      uint32_t a[4];
      const int col = k0 + 2 * t4;
      a[0] = nb[0] >= 0 ? X32[((size_t)nb[0] * cin + col) >> 1] : 0u;
      a[1] = nb[1] >= 0 ? X32[((size_t)nb[1] * cin + col) >> 1] : 0u;
      a[2] = nb[0] >= 0 ? X32[((size_t)nb[0] * cin + col + 8) >> 1] : 0u;
      a[3] = nb[1] >= 0 ? X32[((size_t)nb[1] * cin + col + 8) >> 1] : 0u;
#pragma unroll
      for (int n = 0; n < NT; ++n) {
        // B fragment (16 channels x 8 outputs): W[t][n*8 + g][col], [col + 8]
        const size_t wb = ((size_t)t * COUT + n * 8 + g) * cin + col;
        uint32_t b[2];
        b[0] = __ldg(W32 + (wb >> 1));
        b[1] = __ldg(W32 + ((wb + 8) >> 1));
        mma_bf16(acc[n], a, b);
      }
    }
  }
  // accumulator q: row g + 8 (q >> 1), column 2 t4 + (q & 1)
#pragma unroll
  for (int n = 0; n < NT; ++n) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int h = q >> 1;
      if (row[h] < 0) continue;
      const int co = n * 8 + 2 * t4 + (q & 1);
      float v = acc[n][q] + (bias ? bias[co] : 0.f);
      if (RELU) v = fmaxf(v, 0.f);
      Y[(size_t)row[h] * COUT + co] = __float2bfloat16(v);
    }
  }
}

// dW[t][co][ci] += sum over the block's cells of dY[cell][co] X[nb(cell, t)][ci].
// grid: (cell chunks, 27 taps, ceil(items / 4)); one warp per item = (16 co,
// 16 ci) tile.  A = dY^T (16 co x 16 cells), B = X_t (16 cells x 8 ci).
__global__ void __launch_bounds__(128) k_wgrad(const bf16* __restrict__ dY, int cout,
                                               const bf16* __restrict__ X, int cin,
                                               float* __restrict__ dW, Dims d, int chunk) {
  const int ncell = d.nx * d.ny * d.nz;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int g = lane >> 2, t4 = lane & 3;
  const int t = blockIdx.y;
  const int ci_tiles = cin / 16;
  const int item = blockIdx.z * 4 + wid;
  if (item >= (cout / 16) * ci_tiles) return;
  const int co0 = (item / ci_tiles) * 16, ci0 = (item % ci_tiles) * 16;
  const int cell_begin = blockIdx.x * chunk;
  const int cell_end = min(ncell, cell_begin + chunk);
  float acc[2][4];
#pragma unroll
  for (int n = 0; n < 2; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[n][q] = 0.f;
  const bf16 zero = __float2bfloat16(0.f);
  for (int c0 = cell_begin; c0 < cell_end; c0 += 16) {
    const int cell[4] = {c0 + 2 * t4, c0 + 2 * t4 + 1, c0 + 2 * t4 + 8, c0 + 2 * t4 + 9};
    bf16 lo[4], hi[4];
    int nb[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const bool ok = cell[q] < cell_end;
      lo[q] = ok ? dY[(size_t)cell[q] * cout + co0 + g] : zero;
      hi[q] = ok ? dY[(size_t)cell[q] * cout + co0 + g + 8] : zero;
      const int c = ok ? cell[q] : 0;
      nb[q] = ok ? neighbour(d, c % d.nx, (c / d.nx) % d.ny, c / (d.nx * d.ny), t) : -1;
    }
    uint32_t a[4];
    a[0] = pack2(lo[0], lo[1]);   // row g,     cells 2t4, 2t4+1
    a[1] = pack2(hi[0], hi[1]);   // row g + 8
    a[2] = pack2(lo[2], lo[3]);   // row g,     cells 2t4+8, 2t4+9
    a[3] = pack2(hi[2], hi[3]);   // row g + 8
#pragma unroll
    for (int n = 0; n < 2; ++n) {
      const int c = ci0 + n * 8 + g;
      bf16 x[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = nb[q] >= 0 ? X[(size_t)nb[q] * cin + c] : zero;
      uint32_t b[2];
      b[0] = pack2(x[0], x[1]);
      b[1] = pack2(x[2], x[3]);
      mma_bf16(acc[n], a, b);
    }
  }
#pragma unroll
  for (int n = 0; n < 2; ++n)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int co = co0 + g + 8 * (q >> 1);
      const int c = ci0 + n * 8 + 2 * t4 + (q & 1);
      atomicAdd(dW + ((size_t)t * cout + co) * cin + c, acc[n][q]);
    }
}

// weights of the data-gradient convolution: Wt[26 - t][ci][co] = W[t][co][ci]
__global__ void k_flip(const bf16* __restrict__ W, bf16* __restrict__ Wt, int cout, int cin) {
  const int n = 27 * cout * cin;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int t = e / (cout * cin), rem = e % (cout * cin);
    const int co = rem / cin, c = rem % cin;
    Wt[((size_t)(26 - t) * cin + c) * cout + co] = W[e];
  }
}

// g[e] = 0 where the ReLU output y[e] is not positive
__global__ void k_relu_mask(bf16* __restrict__ g, const bf16* __restrict__ y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    if (!(__bfloat162float(y[e]) > 0.f)) g[e] = __float2bfloat16(0.f);
}

// 2x2x2 mean pooling of X (fine dims d, ch channels) into Y (coarse)
__global__ void k_pool(const bf16* __restrict__ X, bf16* __restrict__ Y, int ch, Dims d) {
  const int cx = d.nx / 2, cy = d.ny / 2, cz = d.nz / 2;
  const int64_t n = (int64_t)cx * cy * cz * ch;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / ch), k = (int)(e % ch);
    const int i = c % cx, j = (c / cx) % cy, l = c / (cx * cy);
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int f = ((2 * l + (q >> 2)) * d.ny + 2 * j + ((q >> 1) & 1)) * d.nx + 2 * i + (q & 1);
      s += __bfloat162float(X[(size_t)f * ch + k]);
    }
    Y[e] = __float2bfloat16(0.125f * s);
  }
}

// adjoint of the pooling, added to dX (fine): dX[f] = dX[f] + dY[coarse(f)] / 8
__global__ void k_pool_back(const bf16* __restrict__ dY, bf16* __restrict__ dX, int ch, Dims d) {
  const int64_t n = (int64_t)d.nx * d.ny * d.nz * ch;
  const int cx = d.nx / 2, cy = d.ny / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / ch), k = (int)(e % ch);
    const int i = f % d.nx, j = (f / d.nx) % d.ny, l = f / (d.nx * d.ny);
    const int c = ((l / 2) * cy + j / 2) * cx + i / 2;
    dX[e] = __float2bfloat16(__bfloat162float(dX[e]) + 0.125f * __bfloat162float(dY[(size_t)c * ch + k]));
  }
}

// decoder input: Y[f] = [X_low[coarse(f)] (lowc ch), S[f] (skipc ch)]
__global__ void k_up_cat(const bf16* __restrict__ Xl, int lowc, const bf16* __restrict__ S,
                         int skipc, bf16* __restrict__ Y, Dims d) {
  const int ch = lowc + skipc;
  const int64_t n = (int64_t)d.nx * d.ny * d.nz * ch;
  const int cx = d.nx / 2, cy = d.ny / 2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int f = (int)(e / ch), k = (int)(e % ch);
    if (k < lowc) {
      const int i = f % d.nx, j = (f / d.nx) % d.ny, l = f / (d.nx * d.ny);
      const int c = ((l / 2) * cy + j / 2) * cx + i / 2;
      Y[e] = Xl[(size_t)c * lowc + k];
    } else {
      Y[e] = S[(size_t)f * skipc + k - lowc];
    }
  }
}

// adjoint of k_up_cat: dXl[c] = sum of the 8 fine gradients (first lowc
// channels), dS[f] = the remaining channels
__global__ void k_up_cat_back(const bf16* __restrict__ dY, int lowc, int skipc,
                              bf16* __restrict__ dXl, bf16* __restrict__ dS, Dims d) {
  const int ch = lowc + skipc;
  const int cx = d.nx / 2, cy = d.ny / 2, cz = d.nz / 2;
  const int64_t nc = (int64_t)cx * cy * cz * lowc;
  const int64_t nf = (int64_t)d.nx * d.ny * d.nz * skipc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nc + nf; e += (int64_t)gridDim.x * blockDim.x) {
    if (e < nc) {
      const int c = (int)(e / lowc), k = (int)(e % lowc);
      const int i = c % cx, j = (c / cx) % cy, l = c / (cx * cy);
      float s = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int f = ((2 * l + (q >> 2)) * d.ny + 2 * j + ((q >> 1) & 1)) * d.nx + 2 * i + (q & 1);
        s += __bfloat162float(dY[(size_t)f * ch + k]);
      }
      dXl[e] = __float2bfloat16(s);
    } else {
      const int64_t e2 = e - nc;
      const int f = (int)(e2 / skipc), k = (int)(e2 % skipc);
      dS[e2] = dY[(size_t)f * ch + lowc + k];
    }
  }
}

// raw input planes in[4][ncell] (float32) -> X[ncell][16] (channels 4..15 zero)
__global__ void k_pack_planes(const float* __restrict__ in, bf16* __restrict__ X, int ncell) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
#pragma unroll
    for (int k = 0; k < 16; ++k)
      X[(size_t)c * 16 + k] = __float2bfloat16(k < 4 ? in[(size_t)k * ncell + c] : 0.f);
}

// max |r| (non-negative floats order like their bit patterns)
__global__ void k_absmax(const float* __restrict__ r, int64_t n, unsigned* out) {
  float m = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(r[e]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// local cell scale h_c^2 = (dx_i dy_j dz_k)^(2/3): r h^2 is the right-hand
// side of the pressure equation in index units (unit spacing)
__device__ __forceinline__ float cell_h2(int c, int nx, int ny, const float* idx0, const float* idx1,
                                         const float* idx2) {
  const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
  return cbrtf(1.f / (idx0[i] * idx1[j] * idx2[k]));
}

// red[2] += sum (r h^2)^2
__global__ void k_rhs_sumsq(const float* __restrict__ r, int nx, int ny, int nz,
                            const float* __restrict__ idx0, const float* __restrict__ idx1,
                            const float* __restrict__ idx2, double* red) {
  const int ncell = nx * ny * nz;
  double s = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const float hh = cell_h2(c, nx, ny, idx0, idx1, idx2);
    const double q = (double)r[c] * (double)(hh * hh);
    s += q * q;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(red + 2, s);
}

// solver input: X[c] = [q_c / S, log(n_x dx_i), log(n_y dy_j), log(n_z dz_k), 0...],
// q = r h^2, S = rms(q) (written to *scale; 0 when r = 0)
__global__ void k_pack_rhs(const float* __restrict__ r, const double* __restrict__ red, int nx,
                           int ny, int nz, const float* __restrict__ idx0,
                           const float* __restrict__ idx1, const float* __restrict__ idx2,
                           bf16* __restrict__ X, float* __restrict__ scale) {
  const int ncell = nx * ny * nz;
  const float S = (float)sqrt(red[2] / ncell);
  const float inv = S > 0.f ? 1.f / S : 0.f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale = S;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
    const float hh = cell_h2(c, nx, ny, idx0, idx1, idx2);
    bf16* o = X + (size_t)c * 16;
    o[0] = __float2bfloat16(r[c] * (hh * hh) * inv);
    o[1] = __float2bfloat16(logf(nx / idx0[i]));
    o[2] = __float2bfloat16(logf(ny / idx1[j]));
    o[3] = __float2bfloat16(logf(nz / idx2[k]));
#pragma unroll
    for (int q = 4; q < 16; ++q) o[q] = __float2bfloat16(0.f);
  }
}

// phi[c] = out[c] * S  (undo the normalisation of input and target)
__global__ void k_unscale(const float* __restrict__ out, const float* __restrict__ scale,
                          float* __restrict__ phi, int n) {
  const float m = *scale;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) phi[c] = out[c] * m;
}

// normalised training target t[c] = phi[c] / S
__global__ void k_scale_target(const double* __restrict__ phi, const float* __restrict__ scale,
                               float* __restrict__ t, int n) {
  const float m = *scale;
  const float s = m > 0.f ? 1.f / m : 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    t[c] = (float)phi[c] * s;
}

__global__ void k_to_f32(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = (float)a[e];
}

// output layer: out[c] = b + sum_k w[k] H[c][k]
__global__ void k_head(const bf16* __restrict__ H, const float* __restrict__ w,
                       const float* __restrict__ b, float* __restrict__ out, int ncell) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    float s = b[0];
#pragma unroll
    for (int k = 0; k < 16; ++k) s += w[k] * __bfloat162float(H[(size_t)c * 16 + k]);
    out[c] = s;
  }
}

// red[0] += sum (out - t)
__global__ void k_err_sum(const float* __restrict__ out, const float* __restrict__ t, int n,
                          double* red) {
  double s = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x)
    s += (double)out[c] - (double)t[c];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(red, s);
}

// mean-free square loss L = mean (e - mean e)^2, e = out - t.  red[1] += L,
// dH = dL/dout * w (BF16), dw[k] += sum dL/dout H[k], db += sum dL/dout.
__global__ void k_head_back(const bf16* __restrict__ H, const float* __restrict__ w,
                            const float* __restrict__ out, const float* __restrict__ t, int n,
                            double* red, bf16* __restrict__ dH, float* __restrict__ dw,
                            float* __restrict__ db) {
  __shared__ float sg[17];
  if (threadIdx.x < 17) sg[threadIdx.x] = 0.f;
  __syncthreads();
  const double ebar = red[0] / n;
  double l = 0.0;
  float gw[16], gb = 0.f;
#pragma unroll
  for (int k = 0; k < 16; ++k) gw[k] = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
    const double e = (double)out[c] - (double)t[c] - ebar;
    l += e * e / n;
    const float go = (float)(2.0 * e / n);
    gb += go;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      gw[k] += go * __bfloat162float(H[(size_t)c * 16 + k]);
      dH[(size_t)c * 16 + k] = __float2bfloat16(go * w[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < 16; ++k) atomicAdd(&sg[k], gw[k]);
  atomicAdd(&sg[16], gb);
  for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(red + 1, l);
  __syncthreads();
  if (threadIdx.x < 16) atomicAdd(dw + threadIdx.x, sg[threadIdx.x]);
  if (threadIdx.x == 16) atomicAdd(db, sg[16]);
}

// db[co] += sum_cells dY[cell][co]; grid (blocks, cout)
__global__ void k_bias_grad(const bf16* __restrict__ dY, int cout, int ncell, float* __restrict__ db) {
  const int co = blockIdx.y;
  float s = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x)
    s += __bfloat162float(dY[(size_t)c * cout + co]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(db + co, s);
}

// Adam (Kingma & Ba 2015) on the float32 parameters; refreshes the BF16 mirror
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ gr, float* __restrict__ m,
                       float* __restrict__ v, bf16* __restrict__ pb, int n, float lr, float b1,
                       float b2, float c1, float c2) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const float g = gr[e];
    const float mm = b1 * m[e] + (1.f - b1) * g;
    const float vv = b2 * v[e] + (1.f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    const float q = p[e] - lr * (mm / c1) / (sqrtf(vv / c2) + 1e-8f);
    p[e] = q;
    pb[e] = __float2bfloat16(q);
  }
}

__global__ void k_mirror(const float* __restrict__ a, bf16* __restrict__ b, int n) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
    b[e] = __float2bfloat16(a[e]);
}

inline unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  b = std::min<int64_t>(b, 152 * 16);
  return (unsigned)std::max<int64_t>(b, 1);
}

}  // namespace unet
}  // namespace fv

struct fv_unet {
  cudaStream_t stream = nullptr;
  int nparam = 0;
  int woff[fv::unet::kNConv] = {}, boff[fv::unet::kNConv] = {};
  int head_w = 0, head_b = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // params, grads, Adam moments
  fv::unet::bf16* pb = nullptr;   // BF16 mirror of the parameters
  fv::unet::bf16* wt = nullptr;   // flipped weights of one layer
  int step = 0;
  // activation workspace, sized for cap cells at level 0 (level l: cap / 8^l)
  int64_t cap = 0, gcap = 0;
  int n[4][3] = {};
  int64_t ncell[4] = {};
  bool have_fwd = false;          // a forward pass at the current dims is in the buffers
  fv::unet::bf16* in16 = nullptr;
  fv::unet::bf16* act[fv::unet::kNConv] = {};
  fv::unet::bf16* cat[3] = {};    // decoder inputs at levels 2, 1, 0
  fv::unet::bf16* pool[3] = {};   // pooled encoder outputs (inputs of levels 1..3)
  float* out = nullptr;           // network output [cells]
  float* tgt = nullptr;           // normalised target [cells]
  double* red = nullptr;          // reductions: loss (0, 1), right-hand side (2)
  float* scale = nullptr;         // normalisation S of the last packed right-hand side
  // gradient workspace (allocated by the first backward pass)
  fv::unet::bf16 *gA = nullptr, *gB = nullptr, *gC = nullptr;
  fv::unet::bf16* gS[3] = {};
};

namespace fv {
namespace unet {

static fv_status dalloc(void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    *p = nullptr;
    set_error("unet: device allocation failed");
    return FV_ENOMEM;
  }
  return FV_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

static void free_ws(fv_unet* u) {
  dfree(u->in16);
  for (auto& a : u->act) { dfree(a); a = nullptr; }
  for (int q = 0; q < 3; ++q) { dfree(u->cat[q]); dfree(u->pool[q]); u->cat[q] = u->pool[q] = nullptr; }
  dfree(u->out); dfree(u->tgt);
  u->in16 = nullptr; u->out = u->tgt = nullptr;
  u->cap = 0;
  u->have_fwd = false;
}

static void free_grad(fv_unet* u) {
  dfree(u->gA); dfree(u->gB); dfree(u->gC);
  u->gA = u->gB = u->gC = nullptr;
  for (auto& s : u->gS) { dfree(s); s = nullptr; }
  u->gcap = 0;
}

static bool dims_ok(int nx, int ny, int nz) {
  auto ok = [](int v) { return v >= 8 && v <= 1024 && v % 8 == 0; };
  return ok(nx) && ok(ny) && ok(nz) && (int64_t)nx * ny * nz <= (int64_t)1 << 27;
}

// set the level dims and make sure the activation buffers hold them
static fv_status ensure_ws(fv_unet* u, int nx, int ny, int nz) {
  if (!dims_ok(nx, ny, nz)) {
    set_error("unet: every dimension must be a multiple of 8 in [8, 1024], at most 2^27 cells");
    return FV_EINVAL;
  }
  const int64_t nc = (int64_t)nx * ny * nz;
  if (nc > u->cap) {
    free_ws(u);
    free_grad(u);
    fv_status s = FV_OK;
    auto A = [&](void** p, size_t b) { if (s == FV_OK) s = dalloc(p, b); };
    A((void**)&u->in16, (size_t)nc * 16 * sizeof(bf16));
    for (int c = 0; c < kNConv; ++c)
      A((void**)&u->act[c], (size_t)(nc >> (3 * kConvs[c].level)) * kConvs[c].cout * sizeof(bf16));
    for (int q = 0; q < 3; ++q) {
      A((void**)&u->cat[q], (size_t)(nc >> (3 * (2 - q))) * kConvs[8 + 2 * q].cin * sizeof(bf16));
      A((void**)&u->pool[q], (size_t)(nc >> (3 * (q + 1))) * kConvs[2 * q + 1].cout * sizeof(bf16));
    }
    A((void**)&u->out, (size_t)nc * sizeof(float));
    A((void**)&u->tgt, (size_t)nc * sizeof(float));
    if (s != FV_OK) { free_ws(u); return s; }
    u->cap = nc;
  }
  const int d[3] = {nx, ny, nz};
  bool same = true;
  for (int a = 0; a < 3; ++a) same = same && u->n[0][a] == d[a];
  for (int l = 0; l < 4; ++l) {
    for (int a = 0; a < 3; ++a) u->n[l][a] = d[a] >> l;
    u->ncell[l] = nc >> (3 * l);
  }
  if (!same) u->have_fwd = false;
  return FV_OK;
}

// Gradient buffers: gA/gB hold one layer's output gradient (at most 16
// channels at level 0; a level l >= 1 holds at most 112 channels on 1/8^l
// of the cells), gC the decoder-input gradient (at most 48 channels at
// level 0), gS[l] the skip gradient of encoder level l.
static fv_status ensure_grad(fv_unet* u) {
  const int64_t nc = u->cap;
  if (u->gcap >= nc) return FV_OK;
  free_grad(u);
  fv_status s = FV_OK;
  auto A = [&](void** p, size_t b) { if (s == FV_OK) s = dalloc(p, b); };
  A((void**)&u->gA, (size_t)nc * 16 * sizeof(bf16));
  A((void**)&u->gB, (size_t)nc * 16 * sizeof(bf16));
  A((void**)&u->gC, (size_t)nc * 48 * sizeof(bf16));
  for (int l = 0; l < 3; ++l) A((void**)&u->gS[l], (size_t)(nc >> (3 * l)) * kConvs[2 * l + 1].cout * sizeof(bf16));
  if (s != FV_OK) { free_grad(u); return s; }
  u->gcap = nc;
  return FV_OK;
}

#define UNET_LAUNCH(...)   \
  do {                     \
    ::fv::count_launch();  \
    __VA_ARGS__;           \
    FV_CHECK_LAUNCH();     \
  } while (0)

template <int COUT, bool RELU>
static fv_status conv_t(cudaStream_t st, const bf16* X, int cin, const bf16* W, const float* b,
                        bf16* Y, const int n[3]) {
  const Dims d{n[0], n[1], n[2]};
  const int64_t warps = ((int64_t)n[0] * n[1] * n[2] + 15) / 16;
  UNET_LAUNCH((k_conv3<COUT, RELU><<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(X, cin, W, b, Y, d)));
  return FV_OK;
}

template <bool RELU>
static fv_status conv(cudaStream_t st, const bf16* X, int cin, const bf16* W, const float* b,
                      bf16* Y, int cout, const int n[3]) {
  switch (cout) {
    case 16: return conv_t<16, RELU>(st, X, cin, W, b, Y, n);
    case 32: return conv_t<32, RELU>(st, X, cin, W, b, Y, n);
    case 48: return conv_t<48, RELU>(st, X, cin, W, b, Y, n);
    case 64: return conv_t<64, RELU>(st, X, cin, W, b, Y, n);
    case 80: return conv_t<80, RELU>(st, X, cin, W, b, Y, n);
    case 112: return conv_t<112, RELU>(st, X, cin, W, b, Y, n);
    default: set_error("unet: unsupported channel count"); return FV_EINVAL;
  }
}

// forward pass from u->in16 to u->out
static fv_status forward(fv_unet* u) {
  cudaStream_t st = u->stream;
  const bf16* X = u->in16;
  for (int l = 0; l < 4; ++l) {
    const int c1 = 2 * l, c2 = 2 * l + 1;
    FV_TRY(conv<true>(st, X, kConvs[c1].cin, u->pb + u->woff[c1], u->p + u->boff[c1], u->act[c1],
                      kConvs[c1].cout, u->n[l]));
    FV_TRY(conv<true>(st, u->act[c1], kConvs[c2].cin, u->pb + u->woff[c2], u->p + u->boff[c2],
                      u->act[c2], kConvs[c2].cout, u->n[l]));
    if (l < 3) {
      const Dims d{u->n[l][0], u->n[l][1], u->n[l][2]};
      UNET_LAUNCH((k_pool<<<blocks_for(u->ncell[l + 1] * kConvs[c2].cout), 256, 0, st>>>(
          u->act[c2], u->pool[l], kConvs[c2].cout, d)));
      X = u->pool[l];
    }
  }
  const bf16* low = u->act[7];
  int lowc = kConvs[7].cout;
  for (int q = 0; q < 3; ++q) {
    const int l = 2 - q, c1 = 8 + 2 * q, c2 = 9 + 2 * q;
    const int skipc = kConvs[2 * l + 1].cout;
    const Dims d{u->n[l][0], u->n[l][1], u->n[l][2]};
    UNET_LAUNCH((k_up_cat<<<blocks_for(u->ncell[l] * (lowc + skipc)), 256, 0, st>>>(
        low, lowc, u->act[2 * l + 1], skipc, u->cat[q], d)));
    FV_TRY(conv<true>(st, u->cat[q], kConvs[c1].cin, u->pb + u->woff[c1], u->p + u->boff[c1],
                      u->act[c1], kConvs[c1].cout, u->n[l]));
    FV_TRY(conv<true>(st, u->act[c1], kConvs[c2].cin, u->pb + u->woff[c2], u->p + u->boff[c2],
                      u->act[c2], kConvs[c2].cout, u->n[l]));
    low = u->act[c2];
    lowc = kConvs[c2].cout;
  }
  UNET_LAUNCH((k_head<<<blocks_for(u->ncell[0]), 256, 0, st>>>(u->act[13], u->p + u->head_w,
                                                                 u->p + u->head_b, u->out,
                                                                 (int)u->ncell[0])));
  u->have_fwd = true;
  return FV_OK;
}

static fv_status relu_back(fv_unet* u, bf16* gy, int c) {
  const int64_t n = u->ncell[kConvs[c].level] * kConvs[c].cout;
  UNET_LAUNCH((k_relu_mask<<<blocks_for(n), 256, 0, u->stream>>>(gy, u->act[c], n)));
  return FV_OK;
}

// parameter gradients of layer c from its pre-activation gradient gy and input X
static fv_status param_grad(fv_unet* u, int c, const bf16* gy, const bf16* X) {
  const ConvSpec& s = kConvs[c];
  const int64_t nc = u->ncell[s.level];
  const Dims d{u->n[s.level][0], u->n[s.level][1], u->n[s.level][2]};
  const int items = (s.cout / 16) * (s.cin / 16);
  const int zb = (items + 3) / 4;
  // about 8 blocks per SM over (chunks x 27 taps x zb), chunks of >= 256 cells
  int64_t chunks = std::max<int64_t>(1, (152 * 8 + 27 * zb - 1) / (27 * zb));
  chunks = std::min<int64_t>(chunks, std::max<int64_t>(1, nc / 256));
  const int64_t chunk = ((nc + chunks - 1) / chunks + 15) / 16 * 16;
  chunks = (nc + chunk - 1) / chunk;
  UNET_LAUNCH((k_wgrad<<<dim3((unsigned)chunks, 27, zb), 128, 0, u->stream>>>(
      gy, s.cout, X, s.cin, u->g + u->woff[c], d, (int)chunk)));
  UNET_LAUNCH((k_bias_grad<<<dim3(std::min<unsigned>(64, blocks_for(nc)), s.cout), 256, 0, u->stream>>>(
      gy, s.cout, (int)nc, u->g + u->boff[c])));
  return FV_OK;
}

// input gradient of layer c: dX = conv(gy, flipped W) (cin channels)
static fv_status data_grad(fv_unet* u, int c, const bf16* gy, bf16* dX) {
  const ConvSpec& s = kConvs[c];
  UNET_LAUNCH((k_flip<<<blocks_for(27 * s.cin * s.cout), 256, 0, u->stream>>>(u->pb + u->woff[c], u->wt,
                                                                               s.cout, s.cin)));
  return conv<false>(u->stream, gy, s.cout, u->wt, nullptr, dX, s.cin, u->n[s.level]);
}

// loss of the last forward pass against u->tgt and all parameter gradients
static fv_status backward(fv_unet* u, double* loss) {
  if (!u->have_fwd) { set_error("unet: backward needs a forward pass at the same dims"); return FV_EINVAL; }
  FV_TRY(ensure_grad(u));
  cudaStream_t st = u->stream;
  const int n0 = (int)u->ncell[0];
  FV_CUDA(cudaMemsetAsync(u->g, 0, u->nparam * sizeof(float), st));
  FV_CUDA(cudaMemsetAsync(u->red, 0, 2 * sizeof(double), st));
  UNET_LAUNCH((k_err_sum<<<blocks_for(n0), 256, 0, st>>>(u->out, u->tgt, n0, u->red)));
  UNET_LAUNCH((k_head_back<<<blocks_for(n0), 256, 0, st>>>(u->act[13], u->p + u->head_w, u->out, u->tgt,
                                                           n0, u->red, u->gA, u->g + u->head_w,
                                                           u->g + u->head_b)));
  bf16* g = u->gA;   // gradient of the current layer's output
  bf16* h = u->gB;
  for (int q = 2; q >= 0; --q) {
    const int l = 2 - q, c1 = 8 + 2 * q, c2 = 9 + 2 * q;
    const int skipc = kConvs[2 * l + 1].cout;
    const int lowc = kConvs[c1].cin - skipc;
    FV_TRY(relu_back(u, g, c2));
    FV_TRY(param_grad(u, c2, g, u->act[c1]));
    FV_TRY(data_grad(u, c2, g, h));
    std::swap(g, h);
    FV_TRY(relu_back(u, g, c1));
    FV_TRY(param_grad(u, c1, g, u->cat[q]));
    FV_TRY(data_grad(u, c1, g, u->gC));
    const Dims d{u->n[l][0], u->n[l][1], u->n[l][2]};
    UNET_LAUNCH((k_up_cat_back<<<blocks_for(u->ncell[l + 1] * lowc + u->ncell[l] * skipc), 256, 0, st>>>(
        u->gC, lowc, skipc, g, u->gS[l], d)));
  }
  for (int l = 3; l >= 0; --l) {
    const int c1 = 2 * l, c2 = 2 * l + 1;
    if (l < 3) {
      // act[c2] feeds the pooling (gradient g, coarse) and the skip (gS[l])
      const Dims d{u->n[l][0], u->n[l][1], u->n[l][2]};
      const int ch = kConvs[c2].cout;
      FV_CUDA(cudaMemcpyAsync(h, u->gS[l], (size_t)u->ncell[l] * ch * sizeof(bf16), cudaMemcpyDeviceToDevice, st));
      UNET_LAUNCH((k_pool_back<<<blocks_for(u->ncell[l] * ch), 256, 0, st>>>(g, h, ch, d)));
      std::swap(g, h);
    }
    const bf16* X = l == 0 ? u->in16 : u->pool[l - 1];
    FV_TRY(relu_back(u, g, c2));
    FV_TRY(param_grad(u, c2, g, u->act[c1]));
    FV_TRY(data_grad(u, c2, g, h));
    std::swap(g, h);
    FV_TRY(relu_back(u, g, c1));
    FV_TRY(param_grad(u, c1, g, X));
    if (l > 0) {
      FV_TRY(data_grad(u, c1, g, h));
      std::swap(g, h);
    }
  }
  if (loss) {
    double hr[2];
    FV_CUDA(cudaMemcpyAsync(hr, u->red, sizeof(hr), cudaMemcpyDeviceToHost, st));
    FV_CUDA(cudaStreamSynchronize(st));
    *loss = hr[1];
  }
  return FV_OK;
}

static fv_status adam(fv_unet* u, float lr) {
  u->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - std::pow(b1, (float)u->step), c2 = 1.f - std::pow(b2, (float)u->step);
  UNET_LAUNCH((k_adam<<<blocks_for(u->nparam), 256, 0, u->stream>>>(u->p, u->g, u->m, u->v, u->pb,
                                                                     u->nparam, lr, b1, b2, c1, c2)));
  return FV_OK;
}

// normalised input of the float32 right-hand side r on grid g into u->in16
// (and its scale S into u->scale)
static fv_status pack_rhs(fv_unet* u, const fv_grid* g, const float* r) {
  cudaStream_t st = u->stream;
  const float* const* idx = g->met_f.idx;
  FV_CUDA(cudaMemsetAsync(u->red + 2, 0, sizeof(double), st));
  UNET_LAUNCH((k_rhs_sumsq<<<blocks_for(g->ncell), 256, 0, st>>>(r, g->n[0], g->n[1], g->n[2], idx[0],
                                                                 idx[1], idx[2], u->red)));
  UNET_LAUNCH((k_pack_rhs<<<blocks_for(g->ncell), 256, 0, st>>>(r, u->red, g->n[0], g->n[1], g->n[2],
                                                                idx[0], idx[1], idx[2], u->in16,
                                                                u->scale)));
  return FV_OK;
}

static fv_status guess_body(fv_unet* u, const fv_grid* g, const float* r, float* phi) {
  FV_TRY(ensure_ws(u, g->n[0], g->n[1], g->n[2]));
  FV_TRY(pack_rhs(u, g, r));
  FV_TRY(forward(u));
  UNET_LAUNCH((k_unscale<<<blocks_for(g->ncell), 256, 0, u->stream>>>(u->out, u->scale, phi,
                                                                      (int)g->ncell)));
  return FV_OK;
}

static fv_status train_body(fv_unet* u, const fv_grid* g, const double* r, const double* phi,
                            float lr, double* loss) {
  FV_TRY(ensure_ws(u, g->n[0], g->n[1], g->n[2]));
  cudaStream_t st = u->stream;
  UNET_LAUNCH((k_to_f32<<<blocks_for(g->ncell), 256, 0, st>>>(r, u->out, g->ncell)));
  FV_TRY(pack_rhs(u, g, u->out));
  UNET_LAUNCH((k_scale_target<<<blocks_for(g->ncell), 256, 0, st>>>(phi, u->scale, u->tgt,
                                                                      (int)g->ncell)));
  FV_TRY(forward(u));
  FV_TRY(backward(u, loss));
  return adam(u, lr);
}

}  // namespace unet

// Guess of phi (float32, device) for the float32 right-hand side r on grid g,
// on the grid's stream (the learned first pass of the SIMPLE loop).  r and
// phi may alias: r is read in full before phi is written.
fv_status unet_guess_f32(fv_unet* u, const fv_grid* g, const float* r, float* phi) {
  cudaStream_t keep = u->stream;
  u->stream = g->stream;
  fv_status s = unet::guess_body(u, g, r, phi);
  u->stream = keep;
  return s;
}

fv_status absmax_f32_host(const fv_grid* g, const float* x, int64_t n, double* out) {
  // one unsigned slot at the end of the grid's scalar area
  unsigned* slot = reinterpret_cast<unsigned*>(g->d_scal + kScalars - 1);
  FV_CUDA(cudaMemsetAsync(slot, 0, sizeof(unsigned), g->stream));
  count_launch();
  unet::k_absmax<<<unet::blocks_for(n), 256, 0, g->stream>>>(x, n, slot);
  FV_CHECK_LAUNCH();
  unsigned bits = 0;
  FV_CUDA(cudaMemcpyAsync(&bits, slot, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  float f;
  std::memcpy(&f, &bits, sizeof(f));
  *out = f;
  return FV_OK;
}

}  // namespace fv

using namespace fv::unet;
using fv::set_error;
using fv::cuda_fail;

extern "C" {

void fv_unet_destroy(fv_unet* u) {
  if (!u) return;
  free_ws(u);
  free_grad(u);
  dfree(u->p); dfree(u->g); dfree(u->m); dfree(u->v); dfree(u->pb); dfree(u->wt);
  dfree(u->red); dfree(u->scale);
  delete u;
}

fv_status fv_unet_create(uint64_t seed, void* cuda_stream, fv_unet** out) {
  if (!out) { set_error("fv_unet_create: out is NULL"); return FV_EINVAL; }
  *out = nullptr;
  fv_unet* u = new fv_unet();
  u->stream = (cudaStream_t)cuda_stream;
  int off = 0;
  for (int c = 0; c < kNConv; ++c) {
    u->woff[c] = off;
    off += 27 * kConvs[c].cin * kConvs[c].cout;
    u->boff[c] = off;
    off += kConvs[c].cout;
  }
  u->head_w = off;
  off += 16;
  u->head_b = off;
  off += 1;
  u->nparam = off;
  int wmax = 0;
  for (const ConvSpec& s : kConvs) wmax = std::max(wmax, 27 * s.cin * s.cout);
  fv_status s = FV_OK;
  auto A = [&](void** p, size_t b) { if (s == FV_OK) s = dalloc(p, b); };
  A((void**)&u->p, off * sizeof(float));
  A((void**)&u->g, off * sizeof(float));
  A((void**)&u->m, off * sizeof(float));
  A((void**)&u->v, off * sizeof(float));
  A((void**)&u->pb, off * sizeof(bf16));
  A((void**)&u->wt, wmax * sizeof(bf16));
  A((void**)&u->red, 4 * sizeof(double));
  A((void**)&u->scale, sizeof(float));
  if (s != FV_OK) { fv_unet_destroy(u); return s; }
  // He-normal weights (seeded), zero biases
  std::vector<float> h(off, 0.f);
  std::mt19937_64 rng(seed);
  std::normal_distribution<float> nd(0.f, 1.f);
  for (int c = 0; c < kNConv; ++c) {
    const float sd = std::sqrt(2.f / (27.f * kConvs[c].cin));
    for (int e = 0; e < 27 * kConvs[c].cin * kConvs[c].cout; ++e) h[u->woff[c] + e] = sd * nd(rng);
  }
  for (int k = 0; k < 16; ++k) h[u->head_w + k] = 0.25f * nd(rng);
  cudaError_t e = cudaMemcpy(u->p, h.data(), off * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(u->g, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(u->m, 0, off * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(u->v, 0, off * sizeof(float));
  if (e == cudaSuccess) {
    fv::count_launch();
    k_mirror<<<blocks_for(off), 256, 0, u->stream>>>(u->p, u->pb, off);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
  if (e != cudaSuccess) {
    fv_status r = cuda_fail(e, "fv_unet_create", __FILE__, __LINE__);
    fv_unet_destroy(u);
    return r;
  }
  *out = u;
  return FV_OK;
}

int fv_unet_param_count(const fv_unet* u) { return u ? u->nparam : 0; }

fv_status fv_unet_set_stream(fv_unet* u, void* cuda_stream) {
  if (!u) { set_error("fv_unet_set_stream: NULL network"); return FV_EINVAL; }
  u->stream = (cudaStream_t)cuda_stream;
  return FV_OK;
}

fv_status fv_unet_set_params(fv_unet* u, const float* params) {
  if (!u || !params) { set_error("fv_unet_set_params: NULL argument"); return FV_EINVAL; }
  FV_CUDA(cudaMemcpyAsync(u->p, params, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  UNET_LAUNCH((k_mirror<<<blocks_for(u->nparam), 256, 0, u->stream>>>(u->p, u->pb, u->nparam)));
  FV_CUDA(cudaMemsetAsync(u->m, 0, u->nparam * sizeof(float), u->stream));
  FV_CUDA(cudaMemsetAsync(u->v, 0, u->nparam * sizeof(float), u->stream));
  u->step = 0;
  return FV_OK;
}

fv_status fv_unet_get_params(const fv_unet* u, float* params, float* grads) {
  if (!u) { set_error("fv_unet_get_params: NULL network"); return FV_EINVAL; }
  if (params)
    FV_CUDA(cudaMemcpyAsync(params, u->p, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  if (grads)
    FV_CUDA(cudaMemcpyAsync(grads, u->g, u->nparam * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  return FV_OK;
}

fv_status fv_unet_forward(fv_unet* u, int nx, int ny, int nz, const float* in, float* out) {
  if (!u || !in || !out) { set_error("fv_unet_forward: NULL argument"); return FV_EINVAL; }
  FV_TRY(ensure_ws(u, nx, ny, nz));
  UNET_LAUNCH((k_pack_planes<<<blocks_for(u->ncell[0]), 256, 0, u->stream>>>(in, u->in16, (int)u->ncell[0])));
  FV_TRY(forward(u));
  FV_CUDA(cudaMemcpyAsync(out, u->out, u->ncell[0] * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  return FV_OK;
}

fv_status fv_unet_backward(fv_unet* u, const float* target, double* loss) {
  if (!u || !target) { set_error("fv_unet_backward: NULL argument"); return FV_EINVAL; }
  if (!u->have_fwd) { set_error("fv_unet_backward: no forward pass to differentiate"); return FV_EINVAL; }
  FV_CUDA(cudaMemcpyAsync(u->tgt, target, u->ncell[0] * sizeof(float), cudaMemcpyDeviceToDevice, u->stream));
  return backward(u, loss);
}

fv_status fv_unet_adam(fv_unet* u, float lr) {
  if (!u || !(lr > 0.f)) { set_error("fv_unet_adam: NULL network or lr <= 0"); return FV_EINVAL; }
  return adam(u, lr);
}

fv_status fv_unet_guess(fv_unet* u, const fv_grid* g, const double* r, double* phi) {
  if (!u || !g || !r || !phi) { set_error("fv_unet_guess: NULL argument"); return FV_EINVAL; }
  cudaStream_t keep = u->stream;
  u->stream = g->stream;
  auto body = [&]() -> fv_status {
    FV_TRY(ensure_ws(u, g->n[0], g->n[1], g->n[2]));
    // float32 copy of r and the guess share the target buffer
    UNET_LAUNCH((k_to_f32<<<blocks_for(g->ncell), 256, 0, u->stream>>>(r, u->tgt, g->ncell)));
    FV_TRY(guess_body(u, g, u->tgt, u->tgt));
    return fv::launch_widen_f32(g, u->tgt, phi, g->ncell);
  };
  fv_status s = body();
  u->stream = keep;
  return s;
}

fv_status fv_unet_train_step(fv_unet* u, const fv_grid* g, const double* r, const double* phi,
                             float lr, double* loss) {
  if (!u || !g || !r || !phi || !(lr > 0.f)) {
    set_error("fv_unet_train_step: NULL argument or lr <= 0");
    return FV_EINVAL;
  }
  cudaStream_t keep = u->stream;
  u->stream = g->stream;
  fv_status s = train_body(u, g, r, phi, lr, loss);
  u->stream = keep;
  return s;
}

}  // extern "C"
