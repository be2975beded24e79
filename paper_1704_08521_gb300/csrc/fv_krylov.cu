// Krylov machinery of Section 3: the SIMPLE-like evaluation of a Krylov
// vector (Eqs. 8-10 and the three-step loop), restarted GMRES(m) inside the
// Newton method, and implicitly restarted Arnoldi for the leading
// eigenvalues of Eq. 7.  Vector work (weighted inner products, classical
// Gram-Schmidt applied twice, combinations) runs in FP64 kernels; the m x m
// Hessenberg matrix is handled in FP64 by the small dense routines.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {

namespace {

constexpr int kDotBlocks = 456;      // 3 x 152 SMs (~40 KB of shared memory and <= 85 registers)
constexpr int kDotChunk = 4096;      // elements staged per block iteration
constexpr int kMaxVec = 130;

// Momentum control-volume size of velocity entry e (0 on wall faces).
__device__ __forceinline__ double face_weight(const Met<double>& m, int64_t e) {
  const int64_t nc = m.ncell;
  const int c = (int)(e / nc);
  const int64_t cell = e - c * nc;
  const int i = (int)(cell % m.n[0]);
  const int64_t t = cell / m.n[0];
  const int j = (int)(t % m.n[1]);
  const int k = (int)(t / m.n[1]);
  const int pos = (c == 0) ? i : (c == 1 ? j : k);
  if (pos == 0) return 0.0;
  const double wx = (c == 0) ? m.dc[0][i] : m.dx[0][i];
  const double wy = (c == 1) ? m.dc[1][j] : m.dx[1][j];
  const double wz = (c == 2) ? m.dc[2][k] : m.dx[2][k];
  return wx * wy * wz;
}

__global__ void k_face_weights(Met<double> m, int64_t n, double* __restrict__ W,
                               float2* __restrict__ Wf) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double x = face_weight(m, e);
    W[e] = x;
    const ff s = f64_split_trunc(x);
    Wf[e] = make_float2(s.hi, s.lo);
  }
}

// ---- weighted inner products: partial[v][block] = sum over the block's
// elements of W w V_v.  The elements are cut into chunks of kDotChunk (16
// per thread); block x owns a contiguous run of whole chunks, block y a group
// of vectors (more than one group only when the chunks alone cannot fill the
// GPU).  Each thread keeps W w of its 16 elements in registers, and the chunk
// of every V_v of the group streams through a ring of kDotStages
// shared-memory tiles of a quarter chunk, filled by asynchronous copies
// (cp.async; 16 bytes where the basis is 16-byte aligned), so the next tiles
// are in flight while one is reduced.  FF: float-float products and sums on
// the FP32 pipes (the bases of the mixed and float-float forms; GB300's FP64
// rate is below the HBM rate for one multiply-add per 8-byte element); else
// FP64.
constexpr int kDotPer = kDotChunk / 256;                  // elements per thread per chunk
constexpr int kDotTile = 1024;                            // entries per ring tile
constexpr int kDotStages = 4;
constexpr int kDotTilesPerChunk = kDotChunk / kDotTile;
constexpr int kDotTPer = kDotTile / 256;                  // elements per thread per tile
constexpr size_t kDotSmem = (size_t)kDotStages * kDotTile * 8 + (size_t)8 * kMaxVec * 8;
static_assert(kDotTilesPerChunk == kDotStages, "ring slot = tile index within the chunk");

__device__ __forceinline__ void cpa8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// a basis entry as float-float: doubles are split, float-float pairs are taken as they are
__device__ __forceinline__ ff to_ff(double d) { return f64_split_trunc(d); }
__device__ __forceinline__ ff to_ff(float2 f) { return ff{f.x, f.y}; }
__device__ __forceinline__ void put_ff(double& d, ff s) { d = ff_join(s.hi, s.lo); }
__device__ __forceinline__ void put_ff(float2& d, ff s) { d = make_float2(s.hi, s.lo); }

__device__ __forceinline__ void cpa16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)), "l"(src) : "memory");
}

// VT: the basis entry type, double or (FF only) a float-float pair (hi, lo);
// al16: V and ldv allow 16-byte copies
template <bool FF, typename VT>
__global__ void __launch_bounds__(256, 3) k_dots_pipe(const double* __restrict__ W,
                                                      const float2* __restrict__ Wf,
                                                      const VT* __restrict__ V, int64_t ldv,
                                                      int nvec, const double* __restrict__ w,
                                                      int64_t n, double* __restrict__ partial,
                                                      int al16, int vb) {
  static_assert(sizeof(VT) == 8, "8-byte basis entries");
  // blockIdx.y: the group of vb vectors this block takes (small grids: more
  // blocks than element chunks); partial[v][blockIdx.x] for its vectors only
  const int v0 = blockIdx.y * vb;
  const int v1 = min(nvec, v0 + vb);
  V += (int64_t)v0 * ldv;
  extern __shared__ __align__(16) unsigned char dsm[];
  VT* ring = (VT*)dsm;
  double* wacc = (double*)(dsm + (size_t)kDotStages * kDotTile * 8);   // [8 warps][kMaxVec]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int i = tid; i < 8 * kMaxVec; i += 256) wacc[i] = 0.0;
  // whole chunks per block (the last block also takes the partial one)
  const int64_t nch = (n + kDotChunk - 1) / kDotChunk;
  const int64_t lo = (nch * blockIdx.x / gridDim.x) * kDotChunk;
  const int64_t hi = blockIdx.x + 1 == gridDim.x ? n : (nch * (blockIdx.x + 1) / gridDim.x) * kDotChunk;
  const int nv_ = v1 - v0;
  const int ntile = nv_ * kDotTilesPerChunk;
  for (int64_t e0 = lo; e0 < hi; e0 += kDotChunk) {
    __syncthreads();                                // the previous chunk is consumed
    const bool full = e0 + kDotChunk <= hi;
    const bool fast = full && al16;                 // two unguarded 16-byte copies per thread per tile
    const VT* vchunk = V + e0 + 2 * tid;
    auto issue = [&](int q) {                       // tile q = quarter q % 4 of V_{q / 4}
      if (q < ntile) {
        const int v = q / kDotTilesPerChunk, part = q % kDotTilesPerChunk;
        VT* dst = ring + part * kDotTile;
        if (fast) {
          const VT* src = vchunk + (int64_t)v * ldv + part * kDotTile;
          cpa16(dst + 2 * tid, src);
          cpa16(dst + 2 * tid + kDotTile / 2, src + kDotTile / 2);
        } else {
          const int64_t b = e0 + (int64_t)part * kDotTile;
          const VT* src = V + (int64_t)v * ldv + b;
          for (int i = tid; i < kDotTile; i += 256)
            if (b + i < hi) cpa8(dst + i, src + i);
        }
      }
      cpa_commit();                                 // empty groups keep the count uniform
    };
    for (int q = 0; q < kDotStages - 1; ++q) issue(q);
    // W w of this thread's elements e0 + k 256 + tid, k < kDotPer
    float2 wf[FF ? kDotPer : 1];
    double wd[FF ? 1 : kDotPer];
#pragma unroll
    for (int h = 0; h < kDotPer; h += kDotPer / 2) {    // two batches of loads in flight
      double wv[kDotPer / 2];
#pragma unroll
      for (int u = 0; u < kDotPer / 2; ++u) {
        const int k = h + u;
        const int64_t e = e0 + k * 256 + tid;
        wv[u] = e < hi ? w[e] : 0.0;
        if constexpr (FF) wf[k] = e < hi ? Wf[e] : make_float2(0.0f, 0.0f);
        else wd[k] = e < hi ? W[e] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < kDotPer / 2; ++u) {
        const int k = h + u;
        if constexpr (FF) {
          const ff x = ff_mul(ff{wf[k].x, wf[k].y}, f64_split_trunc(wv[u]));
          wf[k] = make_float2(x.hi, x.lo);
        } else {
          wd[k] *= wv[u];
        }
      }
    }
    for (int v = 0; v < nv_; ++v) {
      ff sf{0.0f, 0.0f};
      double sd = 0.0;
#pragma unroll
      for (int part = 0; part < kDotTilesPerChunk; ++part) {
        issue(v * kDotTilesPerChunk + part + kDotStages - 1);   // into the slot freed at q - 1
        cpa_wait<kDotStages - 1>();                 // this thread's copies of tile q landed
        __syncthreads();                            // everyone's copies of tile q
        const VT* tile = ring + part * kDotTile;
#pragma unroll
        for (int t = 0; t < kDotTPer; ++t) {
          const int i = t * 256 + tid;
          const int k = part * kDotTPer + t;
          if (full || e0 + part * kDotTile + i < hi) {
            if constexpr (FF) ff_mad(sf, ff{wf[k].x, wf[k].y}, to_ff(tile[i]));
            else sd += wd[k] * tile[i];
          }
        }
        __syncthreads();                            // the slot may be refilled
      }
      // per thread the partial sum of 16 products, then across the warp: in
      // float-float on the FP32 pipes (one TwoSum per level; FP64 adds and
      // conversions here would load GB300's slow FP64 pipe once per 2 elements)
      if constexpr (FF) {
        ff t = sf;
        for (int o = 16; o > 0; o >>= 1) {
          const float xh = __shfl_xor_sync(0xffffffffu, t.hi, o);
          const float xl = __shfl_xor_sync(0xffffffffu, t.lo, o);
          ff u = two_sum(t.hi, xh);
          u.lo += t.lo + xl;
          t = fast_two_sum(u.hi, u.lo);
        }
        if (lane == 0) wacc[warp * kMaxVec + v] += (double)t.hi + (double)t.lo;
      } else {
        double r = sd;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
        if (lane == 0) wacc[warp * kMaxVec + v] += r;
      }
    }
  }
  cpa_wait<0>();
  __syncthreads();
  for (int v = tid; v < nv_; v += 256) {
    double t = 0.0;
    for (int q = 0; q < 8; ++q) t += wacc[q * kMaxVec + v];
    partial[(int64_t)(v0 + v) * gridDim.x + blockIdx.x] = t;
  }
}

// vectors per block-y group: enough groups that nblk x groups fills three
// blocks per SM when the element chunks alone do not
inline int dot_group(int nblk, int nvec) {
  const int groups = std::max(1, std::min(nvec, kDotBlocks / std::max(1, nblk)));
  return (nvec + groups - 1) / groups;
}

__global__ void k_reduce_partials(const double* __restrict__ partial, int nblk,
                                  double* __restrict__ out) {
  __shared__ double red[256];
  const int v = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += partial[(int64_t)v * nblk + b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[v] = red[0];
}

// w += sign * sum_v h[v] V_v
__global__ void __launch_bounds__(256) k_update(double* __restrict__ w, const double* __restrict__ V,
                                                int64_t ldv, int nvec, const double* __restrict__ h,
                                                double sign, int64_t n) {
  __shared__ double hs[kMaxVec];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) hs[v] = sign * h[v];
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double s = w[e];
    int v = 0;
    for (; v + 4 <= nvec; v += 4) {
      const double* p = V + (int64_t)v * ldv + e;
      const double a0 = __ldg(p), a1 = __ldg(p + ldv), a2 = __ldg(p + 2 * ldv), a3 = __ldg(p + 3 * ldv);
      s += hs[v] * a0;
      s += hs[v + 1] * a1;
      s += hs[v + 2] * a2;
      s += hs[v + 3] * a3;
    }
    for (; v < nvec; ++v) s += hs[v] * __ldg(V + (int64_t)v * ldv + e);
    w[e] = s;
  }
}

// k_update in float-float arithmetic (see k_dots_pipe): w += sign * sum_v h[v] V_v
template <typename VT>
__global__ void __launch_bounds__(256) k_update_ff(double* __restrict__ w,
                                                   const VT* __restrict__ V, int64_t ldv,
                                                   int nvec, const double* __restrict__ h,
                                                   double sign, int64_t n) {
  __shared__ float2 hs[kMaxVec];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    const ff x = f64_split_trunc(sign * h[v]);
    hs[v] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    ff s = f64_split_trunc(w[e]);
    int v = 0;
    for (; v + 4 <= nvec; v += 4) {
      const VT* p = V + (int64_t)v * ldv + e;
      const VT a[4] = {__ldg(p), __ldg(p + ldv), __ldg(p + 2 * ldv), __ldg(p + 3 * ldv)};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 c = hs[v + q];
        ff_mad(s, ff{c.x, c.y}, to_ff(a[q]));
      }
    }
    for (; v < nvec; ++v) {
      const float2 c = hs[v];
      ff_mad(s, ff{c.x, c.y}, to_ff(__ldg(V + (int64_t)v * ldv + e)));
    }
    w[e] = ff_join(s.hi, s.lo);
  }
}

// k_update_ff for small grids, where one thread per element leaves the GPU
// mostly idle: 64 elements per block, the vectors split over the block's four
// thread rows (v = row, row + 4, ...), the four float-float partial sums
// added in shared memory before w is updated
template <typename VT>
__global__ void __launch_bounds__(256) k_update_vsplit(double* __restrict__ w,
                                                       const VT* __restrict__ V, int64_t ldv,
                                                       int nvec, const double* __restrict__ h,
                                                       double sign, int64_t n) {
  __shared__ float2 hs[kMaxVec];
  __shared__ float2 part[4][64];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    const ff x = f64_split_trunc(sign * h[v]);
    hs[v] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
  const int64_t e = (int64_t)blockIdx.x * 64 + tx;
  ff s{0.0f, 0.0f};
  if (e < n)
    for (int v = ty; v < nvec; v += 4) {
      const float2 c = hs[v];
      ff_mad(s, ff{c.x, c.y}, to_ff(__ldg(V + (int64_t)v * ldv + e)));
    }
  part[ty][tx] = make_float2(s.hi, s.lo);
  __syncthreads();
  if (ty == 0 && e < n) {
    ff t = f64_split_trunc(w[e]);
#pragma unroll
    for (int q = 0; q < 4; ++q) t = ff_add(t, ff{part[q][tx].x, part[q][tx].y});
    w[e] = ff_join(t.hi, t.lo);
  }
}

// grids below this many velocity entries take k_update_vsplit
constexpr int64_t kUpdateSplitBelow = 1 << 20;

// k_update_ff for a float-float basis, two adjacent elements per thread with
// 16-byte loads (w, V and ldv 16-byte aligned / even); the odd last element,
// if any, by the first thread
__global__ void __launch_bounds__(256) k_update_ffb2(double* __restrict__ w,
                                                     const float2* __restrict__ V, int64_t ldv,
                                                     int nvec, const double* __restrict__ h,
                                                     double sign, int64_t n) {
  __shared__ float2 hs[kMaxVec];
  for (int v = threadIdx.x; v < nvec; v += blockDim.x) {
    const ff x = f64_split_trunc(sign * h[v]);
    hs[v] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t np = n / 2;
  for (int64_t pi = gt; pi < np; pi += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = 2 * pi;
    const double2 wv = *reinterpret_cast<const double2*>(w + e);
    ff s0 = f64_split_trunc(wv.x), s1 = f64_split_trunc(wv.y);
    int v = 0;
    for (; v + 4 <= nvec; v += 4) {
      const float2* p = V + (int64_t)v * ldv + e;
      const float4 a[4] = {__ldg(reinterpret_cast<const float4*>(p)),
                           __ldg(reinterpret_cast<const float4*>(p + ldv)),
                           __ldg(reinterpret_cast<const float4*>(p + 2 * ldv)),
                           __ldg(reinterpret_cast<const float4*>(p + 3 * ldv))};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 c = hs[v + q];
        ff_mad(s0, ff{c.x, c.y}, ff{a[q].x, a[q].y});
        ff_mad(s1, ff{c.x, c.y}, ff{a[q].z, a[q].w});
      }
    }
    for (; v < nvec; ++v) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(V + (int64_t)v * ldv + e));
      const float2 c = hs[v];
      ff_mad(s0, ff{c.x, c.y}, ff{a.x, a.y});
      ff_mad(s1, ff{c.x, c.y}, ff{a.z, a.w});
    }
    *reinterpret_cast<double2*>(w + e) = make_double2(ff_join(s0.hi, s0.lo), ff_join(s1.hi, s1.lo));
  }
  if (gt == 0 && (n & 1)) {
    const int64_t e = n - 1;
    ff s = f64_split_trunc(w[e]);
    for (int v = 0; v < nvec; ++v) {
      const float2 c = hs[v];
      ff_mad(s, ff{c.x, c.y}, to_ff(V[(int64_t)v * ldv + e]));
    }
    w[e] = ff_join(s.hi, s.lo);
  }
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b,
                        const double* __restrict__ y, double* __restrict__ out) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = a * x[e] + (y ? b * y[e] : 0.0);
}

// mode 0: out = x / s ; mode 1: out = x * s
__global__ void k_scale_dev(int64_t n, const double* __restrict__ x, const double* __restrict__ s,
                            int mode, double* __restrict__ out) {
  const double f = mode == 0 ? 1.0 / s[0] : s[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = x[e] * f;
}

// out_c = sum_i V_i C[i][c], c < nout; 32 elements per block staged in
// shared memory so out may alias the first columns of V.
__global__ void __launch_bounds__(256) k_combine(const double* V, int64_t ldv, int nin,
                                                 const double* __restrict__ C, int nout,
                                                 double* out, int64_t ldo, int64_t n) {
  extern __shared__ double sv[];   // nin x 32
  const int el = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + el;
  for (int i = grp; i < nin; i += 8) sv[i * 32 + el] = (e < n) ? V[(int64_t)i * ldv + e] : 0.0;
  __syncthreads();
  if (e >= n) return;
  for (int c = grp; c < nout; c += 8) {
    double s = 0.0;
    for (int i = 0; i < nin; ++i) s += sv[i * 32 + el] * __ldg(C + (int64_t)i * nout + c);
    out[(int64_t)c * ldo + e] = s;
  }
}

// k_combine in float-float arithmetic (see k_dots_pipe): the nin x nout
// coefficients are split into shared memory once per block, each block
// stages 32 elements of every input vector as float-float pairs.
template <typename VT, typename OT>
__global__ void __launch_bounds__(256) k_combine_ff(const VT* V, int64_t ldv, int nin,
                                                    const double* __restrict__ C, int nout,
                                                    OT* out, int64_t ldo, int64_t n) {
  extern __shared__ float2 smf[];   // nin x 32 inputs, then nin x nout coefficients
  float2* sv = smf;
  float2* cs = smf + nin * 32;
  const int el = threadIdx.x & 31, grp = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + el;
  for (int i = grp; i < nin; i += 8) {
    ff x{0.0f, 0.0f};
    if (e < n) x = to_ff(V[(int64_t)i * ldv + e]);
    sv[i * 32 + el] = make_float2(x.hi, x.lo);
  }
  for (int q = threadIdx.x; q < nin * nout; q += blockDim.x) {
    const ff x = f64_split_trunc(C[q]);
    cs[q] = make_float2(x.hi, x.lo);
  }
  __syncthreads();
  if (e >= n) return;
  for (int c = grp; c < nout; c += 8) {
    ff s{0.0f, 0.0f};
    for (int i = 0; i < nin; ++i) {
      const float2 a = sv[i * 32 + el], b = cs[i * nout + c];
      ff_mad(s, ff{a.x, a.y}, ff{b.x, b.y});
    }
    put_ff(out[(int64_t)c * ldo + e], s);
  }
}

// basis column <-> double vector: col = split(scale x) / x = join(col)
__global__ void k_store_ff(int64_t n, const double* __restrict__ x, double scale,
                           float2* __restrict__ col) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ff s = f64_split_trunc(scale * x[e]);
    col[e] = make_float2(s.hi, s.lo);
  }
}

__global__ void k_load_ff(int64_t n, const float2* __restrict__ col, double* __restrict__ x) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float2 c = col[e];
    x[e] = ff_join(c.x, c.y);
  }
}

__global__ void k_maxabs(int64_t n, const double* __restrict__ x, double* slot, double* nanslot) {
  __shared__ double red[32];
  double a = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = fabs(x[e]);
    if (!(v <= 1e300)) *nanslot = 1.0;
    else a = fmax(a, v);
  }
  for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x < 32) {
    a = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    if (threadIdx.x == 0)
      atomicMax((unsigned long long*)slot, (unsigned long long)__double_as_longlong(a));
  }
}

__global__ void k_widen(const float* __restrict__ s, double* __restrict__ d, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    d[e] = double(s[e]);
}

inline unsigned grid1d(int64_t n, int per_block = 256) {
  int64_t b = (n + per_block - 1) / per_block;
  return (unsigned)std::min<int64_t>(std::max<int64_t>(b, 1), 152 * 16);
}

}  // namespace

fv_status fill_face_weights(fv_grid* g) {
  // three ~40 KB dot-product blocks per SM
  const void* dk[3] = {(const void*)k_dots_pipe<false, double>, (const void*)k_dots_pipe<true, double>,
                       (const void*)k_dots_pipe<true, float2>};
  for (const void* f : dk) {
    FV_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDotSmem));
    FV_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  }
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_face_weights<<<grid1d(g->nvel), 256, 0, g->stream>>>(g->met_d, g->nvel, g->wts, g->wts_ff);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_dots(const fv_grid* g, const double* V, int64_t ldv, int nvec, const double* w,
                   double* d_out, bool ff_arith) {
  if (nvec <= 0) return FV_OK;
  if (nvec > kMaxVec) { set_error("vec_dots: too many vectors"); return FV_EINVAL; }
  const int64_t n = g->nvel;
  // each block an even share of at least one chunk; two blocks per SM
  const int nblk = (int)std::min<int64_t>(kDotBlocks, (n + kDotChunk - 1) / kDotChunk);
  {
    LaunchScope ls_(g, FV_K_DOTS);
    const int al16 = ((uintptr_t)V % 16 == 0) && (ldv % 2 == 0);
    const int vb = dot_group(nblk, nvec);
    const dim3 grid(nblk, (nvec + vb - 1) / vb);
    if (ff_arith)
      k_dots_pipe<true, double><<<grid, 256, kDotSmem, g->stream>>>(g->wts, g->wts_ff, V, ldv,
                                                                  nvec, w, n, g->d_part, al16, vb);
    else
      k_dots_pipe<false, double><<<grid, 256, kDotSmem, g->stream>>>(g->wts, g->wts_ff, V, ldv,
                                                                   nvec, w, n, g->d_part, al16, vb);
  }
  FV_CHECK_LAUNCH();
  {
    LaunchScope ls_(g, FV_K_DOTS);
    k_reduce_partials<<<nvec, 256, 0, g->stream>>>(g->d_part, nblk, d_out);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_update(const fv_grid* g, double* w, const double* V, int64_t ldv, int nvec,
                     const double* d_h, double sign, bool ff_arith) {
  if (nvec <= 0) return FV_OK;
  if (nvec > kMaxVec) { set_error("vec_update: too many vectors"); return FV_EINVAL; }
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    if (ff_arith && g->nvel < kUpdateSplitBelow)
      k_update_vsplit<double><<<(unsigned)((g->nvel + 63) / 64), 256, 0, g->stream>>>(
          w, V, ldv, nvec, d_h, sign, g->nvel);
    else if (ff_arith)
      k_update_ff<double><<<grid1d(g->nvel), 256, 0, g->stream>>>(w, V, ldv, nvec, d_h, sign,
                                                                  g->nvel);
    else
      k_update<<<grid1d(g->nvel), 256, 0, g->stream>>>(w, V, ldv, nvec, d_h, sign, g->nvel);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_axpby(const fv_grid* g, int64_t n, double a, const double* x, double b,
                    const double* y, double* out) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_axpby<<<grid1d(n), 256, 0, g->stream>>>(n, a, x, b, y, out);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_scale_by_device(const fv_grid* g, int64_t n, const double* x, const double* d_s,
                              int mode, double* out) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_scale_dev<<<grid1d(n), 256, 0, g->stream>>>(n, x, d_s, mode, out);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_combine(const fv_grid* g, const double* V, int64_t ldv, int nin, const double* d_C,
                      int nout, double* out, int64_t ldo, bool ff_arith) {
  const int64_t n = g->nvel;
  const size_t smem = ff_arith ? (size_t)nin * (32 + nout) * sizeof(float2)
                               : (size_t)nin * 32 * sizeof(double);
  if (smem > 200 * 1024) { set_error("vec_combine: too many inputs"); return FV_EINVAL; }
  if (smem > 48 * 1024)
    FV_CUDA(cudaFuncSetAttribute(ff_arith ? (const void*)k_combine_ff<double, double>
                                          : (const void*)k_combine,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    if (ff_arith)
      k_combine_ff<double, double><<<(unsigned)((n + 31) / 32), 256, smem, g->stream>>>(
          V, ldv, nin, d_C, nout, out, ldo, n);
    else
      k_combine<<<(unsigned)((n + 31) / 32), 256, smem, g->stream>>>(V, ldv, nin, d_C, nout, out,
                                                                    ldo, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

// Gram-Schmidt step of a device-resident Arnoldi cycle: column j of H gets
// h_i = (first + second CGS pass coefficients) for i < j1 and the norm of the
// new vector at row j1 (sub_only: the norm alone); *scale = 1 / norm.
__global__ void k_gs_finish(const double* __restrict__ dh1, const double* __restrict__ dh2,
                            const double* __restrict__ dnn, int j1, double* __restrict__ Hcol, int ld,
                            double* __restrict__ scale, int sub_only) {
  if (!sub_only)
    for (int i = threadIdx.x; i < j1; i += blockDim.x) Hcol[(int64_t)i * ld] = dh1[i] + dh2[i];
  if (threadIdx.x == 0) {
    const double hn = sqrt(fmax(dnn[0], 0.0));
    Hcol[(int64_t)j1 * ld] = hn;
    scale[0] = hn > 0.0 ? 1.0 / hn : 0.0;
  }
}

__global__ void k_store_ff_dev(int64_t n, const double* __restrict__ x, const double* __restrict__ scale,
                               float2* __restrict__ col) {
  const double sc = scale[0];
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const ff s = f64_split_trunc(sc * x[e]);
    col[e] = make_float2(s.hi, s.lo);
  }
}

// entry of largest modulus of the complex vector (re, im): per-block
// (value, index) partials, then one block reduces them and writes
// out[0] = re[big], out[1] = im[big]
__global__ void k_absmax_c(int64_t n, const double* __restrict__ re, const double* __restrict__ im,
                           double* __restrict__ pv, int64_t* __restrict__ pi) {
  __shared__ double sv[256];
  __shared__ int64_t si[256];
  double bv = -1.0;
  int64_t bi = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double v = re[e] * re[e] + im[e] * im[e];
    if (v > bv) { bv = v; bi = e; }
  }
  sv[threadIdx.x] = bv;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double o = sv[threadIdx.x + s];
      const int64_t oi = si[threadIdx.x + s];
      if (o > sv[threadIdx.x] || (o == sv[threadIdx.x] && oi < si[threadIdx.x])) {
        sv[threadIdx.x] = o;
        si[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { pv[blockIdx.x] = sv[0]; pi[blockIdx.x] = si[0]; }
}

__global__ void k_absmax_c_final(int nb, const double* __restrict__ pv, const int64_t* __restrict__ pi,
                                 const double* __restrict__ re, const double* __restrict__ im,
                                 double* __restrict__ out) {
  if (threadIdx.x != 0) return;
  double bv = -1.0;
  int64_t bi = 0;
  for (int b = 0; b < nb; ++b)
    if (pv[b] > bv || (pv[b] == bv && pi[b] < bi)) { bv = pv[b]; bi = pi[b]; }
  out[0] = re[bi];
  out[1] = im[bi];
}

// ---- a Krylov basis stored as float-float pairs (the mixed and float-float
// Arnoldi bases): each vector is split once when it is stored, so the
// Gram-Schmidt kernels read (hi, lo) pairs instead of splitting doubles
static fv_status ffb_dots(const fv_grid* g, const float2* Vf, int nvec, const double* w,
                          double* d_out) {
  if (nvec <= 0) return FV_OK;
  if (nvec > kMaxVec) { set_error("ffb_dots: too many vectors"); return FV_EINVAL; }
  const int64_t n = g->nvel;
  const int nblk = (int)std::min<int64_t>(kDotBlocks, (n + kDotChunk - 1) / kDotChunk);
  {
    LaunchScope ls_(g, FV_K_DOTS);
    const int al16 = ((uintptr_t)Vf % 16 == 0) && (n % 2 == 0);
    const int vb = dot_group(nblk, nvec);
    const dim3 grid(nblk, (nvec + vb - 1) / vb);
    k_dots_pipe<true, float2><<<grid, 256, kDotSmem, g->stream>>>(g->wts, g->wts_ff, Vf, n, nvec,
                                                                  w, n, g->d_part, al16, vb);
  }
  FV_CHECK_LAUNCH();
  {
    LaunchScope ls_(g, FV_K_DOTS);
    k_reduce_partials<<<nvec, 256, 0, g->stream>>>(g->d_part, nblk, d_out);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

static fv_status ffb_update(const fv_grid* g, double* w, const float2* Vf, int nvec,
                            const double* d_h, double sign) {
  if (nvec <= 0) return FV_OK;
  if (nvec > kMaxVec) { set_error("ffb_update: too many vectors"); return FV_EINVAL; }
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    const int64_t n = g->nvel;
    if (n < kUpdateSplitBelow)
      k_update_vsplit<float2><<<(unsigned)((n + 63) / 64), 256, 0, g->stream>>>(w, Vf, n, nvec, d_h,
                                                                              sign, n);
    else if ((uintptr_t)w % 16 == 0 && (uintptr_t)Vf % 16 == 0 && n % 2 == 0)
      k_update_ffb2<<<grid1d(n / 2 + 1), 256, 0, g->stream>>>(w, Vf, n, nvec, d_h, sign, n);
    else
      k_update_ff<float2><<<grid1d(n), 256, 0, g->stream>>>(w, Vf, n, nvec, d_h, sign, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

// out_c = sum_i V_i C[i][c] (C: nin x nout on the device, row-major); out is
// a float-float basis (may alias the first columns of Vf) or doubles
template <typename OT>
static fv_status ffb_combine(const fv_grid* g, const float2* Vf, int nin, const double* d_C,
                             int nout, OT* out) {
  const int64_t n = g->nvel;
  const size_t smem = (size_t)nin * (32 + nout) * sizeof(float2);
  if (smem > 200 * 1024) { set_error("ffb_combine: too many inputs"); return FV_EINVAL; }
  if (smem > 48 * 1024)
    FV_CUDA(cudaFuncSetAttribute(k_combine_ff<float2, OT>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_combine_ff<float2, OT><<<(unsigned)((n + 31) / 32), 256, smem, g->stream>>>(
        Vf, n, nin, d_C, nout, out, n, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

static fv_status ffb_store(const fv_grid* g, const double* x, double scale, float2* col) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_store_ff<<<grid1d(g->nvel), 256, 0, g->stream>>>(g->nvel, x, scale, col);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

static fv_status ffb_load(const fv_grid* g, const float2* col, double* x) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_load_ff<<<grid1d(g->nvel), 256, 0, g->stream>>>(g->nvel, col, x);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status vec_maxabs(const fv_grid* g, int64_t n, const double* x, double* slot) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_maxabs<<<grid1d(n), 256, 0, g->stream>>>(n, x, slot, g->d_scal + S_NAN);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status widen_float(const fv_grid* g, const float* src, double* dst, int64_t n) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_widen<<<grid1d(n), 256, 0, g->stream>>>(src, dst, n);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

fv_status reset_scalars(const fv_grid* g) {
  FV_CUDA(cudaMemsetAsync(g->d_scal, 0, kScalars * sizeof(double), g->stream));
  return FV_OK;
}

fv_status fetch_scalars(const fv_grid* g, double* host) {
  FV_CUDA(cudaMemcpyAsync(g->h_scal, g->d_scal, kScalars * sizeof(double), cudaMemcpyDeviceToHost,
                          g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  std::memcpy(host, g->h_scal, kScalars * sizeof(double));
  return FV_OK;
}

double bits_to_double(double slot) { return slot; }

// ------------------------------------------------------------------------
// SIMPLE loop (Section 3): from w in `cur` (overwritten), iterate
//   phi = (D G)^+ D v ; v -= omega G phi ; p += omega phi
// until ||phi_k|| <= eps ||phi_1||.  The result ends in `out` (== cur or
// another buffer of n_vel); `spare` is scratch of n_vel.
struct SimpleResult {
  int passes = 0;
  double phi_first = 0.0, phi_last = 0.0, div_max = 0.0;
};

// mg (FV_FP64 only): each pass solves the pressure correction by multigrid
// to mg->rtol instead of by the tensor-product factorisation
static fv_status simple_loop(const fv_grid* g, double* cur, double* spare, double* out, double* p,
                             double eps, int max_pass, int prec, double omega, SimpleResult* res_out,
                             double div_abs = 0.0, const fv_mg_opts* mg = nullptr) {
  SimpleResult local;
  SimpleResult* res = res_out ? res_out : &local;
  double* r = g->cell_buf[0];
  void* phi = (void*)g->cell_buf[1];
  FV_TRY(reset_scalars(g));
  FV_TRY(launch_divergence(g, cur, r, nullptr));
  if (p) FV_CUDA(cudaMemsetAsync(p, 0, g->ncell * sizeof(double), g->stream));
  double h[kScalars];
  double phi1 = 0.0;
  res->passes = 0;
  fv_status st = FV_ENOCONV;
  for (int pass = 1; pass <= max_pass; ++pass) {
    if (mg) {
      fv_status ms = mg_solve(const_cast<fv_grid*>(g), r, (double*)phi, nullptr, *mg, nullptr);
      if (ms != FV_OK && ms != FV_ENOCONV) return ms;   // a capped inexact solve is corrected later
    } else {
      FV_TRY(tpf_solve(g, r, phi, prec));
    }
    FV_TRY(reset_scalars(g));
    FV_TRY(launch_correct_div(g, cur, spare, phi, prec == FV_MIXED, p, r, omega));
    std::swap(cur, spare);
    FV_TRY(fetch_scalars(g, h));
    res->passes = pass;
    const double ph = h[S_PHI_MAX];
    res->div_max = h[S_DIV_MAX];
    if (h[S_NAN] != 0.0) { set_error("SIMPLE loop: NaN/Inf in the correction"); return FV_ENAN; }
    if (pass == 1) phi1 = ph;
    res->phi_first = phi1;
    const double prev = res->phi_last;
    res->phi_last = ph;
    if (ph == 0.0 || ph <= eps * phi1 || res->div_max <= div_abs) { st = FV_OK; break; }
    // round-off floor: the corrections stopped shrinking at a level far
    // below the first one (the requested eps lies under the floor of the
    // arithmetic); the fields are as divergence-free as they can get
    if (pass >= 3 && ph > 0.25 * prev && ph <= 1e-9 * phi1) { st = FV_OK; break; }
  }
  if (cur != out) FV_CUDA(cudaMemcpyAsync(out, cur, g->nvel * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  if (st != FV_OK) set_error("SIMPLE loop reached max_pass");
  return st;
}

static float slot_float(const double* h, int slot) {
  float f;
  std::memcpy(&f, (const char*)(h + slot), sizeof(float));
  return f;
}

// Mixed-precision SIMPLE loop on the float-float state, starting from the
// float32 predictor in g->w32 whose divergence is in g->r32.  Writes
// out = v - sigma x (float64) and p_out (optional).
// phi_guess (optional): pass 1 takes this float32 phi instead of the exact
// solve; the stop test then refers to max |p| after pass 2 (guess + first
// exact correction), the first exact correction of the plain loop.
static fv_status simple_loop_ff(const fv_grid* g, double* out, double* p_out, const double* x,
                                double sigma, double eps, int max_pass, double omega,
                                SimpleResult* res_out, bool ff_start = false,
                                const float* phi_guess = nullptr) {
  SimpleResult local;
  SimpleResult* res = res_out ? res_out : &local;
  // ff_start: the predictor is the float-float field in vff[1] and p starts at 0
  const void* cur = ff_start ? (const void*)g->vff[1] : (const void*)g->w32;
  if (ff_start) FV_CUDA(cudaMemsetAsync(g->pff, 0, g->ncell * sizeof(float2), g->stream));
  int nxt = 0;
  double h[kScalars];
  double phi1 = 0.0;
  res->passes = 0;
  res->phi_last = 0.0;
  fv_status st = FV_ENOCONV;
  const int first_exact = phi_guess ? 2 : 1;
  for (int pass = 1; pass <= max_pass; ++pass) {
    const float* phi = g->phi32;
    if (pass == 1 && phi_guess) phi = phi_guess;
    else FV_TRY(tpf_solve_f32(g, g->r32, g->phi32));
    FV_TRY(reset_scalars(g));
    FV_TRY(launch_correct_ff(g, pass == 1 && !ff_start, cur, g->vff[nxt], phi, g->pff, g->r32,
                             omega, ff_start));
    cur = g->vff[nxt];
    nxt ^= 1;
    FV_TRY(fetch_scalars(g, h));
    res->passes = pass;
    bool timed_out = false;
    FV_TRY(take_fault(g, &timed_out));
    if (timed_out) return status_error(4);
    if (h[S_NAN] != 0.0) { set_error("SIMPLE loop: NaN/Inf in the correction"); return FV_ENAN; }
    const double ph = slot_float(h, S_PHI_MAX_F);
    res->div_max = slot_float(h, S_DIV_MAX_F);
    const double prev = res->phi_last;
    res->phi_last = ph;
    if (pass < first_exact) continue;   // the guess pass never ends the loop
    if (pass == first_exact) {
      phi1 = ph;
      if (phi_guess) FV_TRY(absmax_f32_host(g, (const float*)g->pff, 2 * g->ncell, &phi1));
    }
    res->phi_first = phi1;
    if (ph == 0.0 || ph <= eps * phi1) { st = FV_OK; break; }
    if (pass >= first_exact + 2 && ph > 0.25 * prev && ph <= 1e-9 * phi1) { st = FV_OK; break; }
  }
  FV_TRY(launch_join_ff(g, (const float2*)cur, sigma != 0.0 ? x : nullptr, sigma, out, g->nvel));
  if (p_out) FV_TRY(launch_join_ff_cells(g, g->pff, p_out));
  if (st != FV_OK) set_error("SIMPLE loop reached max_pass");
  return st;
}

// out = P w32 (the float32 field in g->w32, whose divergence is in g->r32):
// the mixed SIMPLE loop without a predictor, to a relative correction eps
fv_status simple_project_w32(const fv_grid* g, double* out, double eps) {
  SimpleResult r;
  return simple_loop_ff(g, out, nullptr, nullptr, 0.0, eps, 50, 1.0, &r);
}

// A_sigma x = P (L_U x + sigma x) - sigma x  (sigma = 0: the Krylov vector).
// out must not alias x.  Uses vel_buf[0] as scratch.
static fv_status krylov_apply(const fv_grid* g, const double* U, const double* x, double* out,
                              double* p, double sigma, int prec, double eps, int max_pass,
                              double omega, SimpleResult* res) {
  if (prec == FV_MIXED || prec == FV_FF) {
    if (g->use_graph) {
      int status = 0;
      FV_TRY(mixed_krylov_graph(g, U, x, out, p, sigma, eps, max_pass, omega, res != nullptr,
                                res ? &res->passes : nullptr, res ? &res->phi_first : nullptr,
                                res ? &res->phi_last : nullptr, res ? &res->div_max : nullptr,
                                &status, prec));
      return res ? status_error(status) : FV_OK;
    }
    if (prec == FV_FF) {
      FV_TRY(launch_jv_ff(g, U, x, g->vff[1], sigma));
      FV_TRY(launch_div_ff(g, g->vff[1], g->r32));
      return simple_loop_ff(g, out, p, x, sigma, eps, max_pass, omega, res, true);
    }
    FV_TRY(launch_jv_f32(g, U, x, g->w32, sigma));
    FV_TRY(launch_div_f32(g, g->w32, g->r32));
    return simple_loop_ff(g, out, p, x, sigma, eps, max_pass, omega, res);
  }
  FV_TRY(launch_momentum_jac(g, U ? U : g->base_ptr, x, out, prec, sigma));
  fv_status s = simple_loop(g, out, g->vel_buf[0], out, p, eps, max_pass, prec, omega, res);
  if (s != FV_OK) return s;
  if (sigma != 0.0) FV_TRY(vec_axpby(g, g->nvel, 1.0, out, -sigma, x, out));
  return FV_OK;
}

static fv_status maxabs_host(const fv_grid* g, int64_t n, const double* x, double* out, bool* nan);

// The Krylov drivers launch graph evaluations without waiting for their
// status (krylov_apply with res = nullptr) and check, once per cycle, the
// worst status since the last check: the error krylov_apply would have
// returned for any of them.  Host-driven evaluations report at once.
static fv_status check_products(const fv_grid* gc, int prec) {
  fv_grid* g = const_cast<fv_grid*>(gc);
  if (!(g->use_graph && (prec == FV_MIXED || prec == FV_FF))) return FV_OK;
  int w = 0;
  FV_TRY(graph_take_status(g, &w));
  return status_error(w);
}

// Project x in place onto divergence-free fields (p: optional pressure out),
// until the divergence is at round-off level for the size of x.
static fv_status project_inplace(const fv_grid* g, double* x, double* p, int prec, double eps,
                                 SimpleResult* res) {
  double xmax;
  FV_TRY(maxabs_host(g, g->nvel, x, &xmax, nullptr));
  double hmin = 1.0;
  for (int d = 0; d < 3; ++d)
    for (double h : g->h_dx[d]) hmin = std::min(hmin, h);
  return simple_loop(g, x, g->vel_buf[0], x, p, eps, 200, prec, 1.0, res, 1e-14 * xmax / hmin);
}

static fv_status ensure_krylov(fv_grid* g, int cols) {
  if (g->kry && g->kry_cols >= cols) return FV_OK;
  if (g->kry) { cudaFree(g->kry); g->kry = nullptr; }
  if (g->kry_small) { cudaFree(g->kry_small); g->kry_small = nullptr; }
  cudaError_t e = cudaMalloc((void**)&g->kry, (size_t)cols * g->nvel * sizeof(double));
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    set_error("Krylov basis allocation failed");
    return FV_ENOMEM;
  }
  FV_CUDA(cudaMalloc((void**)&g->kry_small, (size_t)(kMaxVec + 2) * (kMaxVec + 2) * sizeof(double)));
  g->kry_cols = cols;
  return FV_OK;
}

// CGS2 of w against V[0..j] in the W-inner product; returns h (j+1) and
// ||w||_W on the host.
static fv_status cgs2(const fv_grid* g, const double* V, int j1, double* w, double* h_host,
                      double* wnorm, bool ff_arith) {
  double* dh1 = g->kry_small;
  double* dh2 = g->kry_small + kMaxVec;
  double* dnn = g->kry_small + 2 * kMaxVec;
  FV_TRY(vec_dots(g, V, g->nvel, j1, w, dh1, ff_arith));
  FV_TRY(vec_update(g, w, V, g->nvel, j1, dh1, -1.0, ff_arith));
  FV_TRY(vec_dots(g, V, g->nvel, j1, w, dh2, ff_arith));
  FV_TRY(vec_update(g, w, V, g->nvel, j1, dh2, -1.0, ff_arith));
  FV_TRY(vec_dots(g, w, g->nvel, 1, w, dnn, ff_arith));
  std::vector<double> tmp(2 * kMaxVec + 1);
  FV_CUDA(cudaMemcpyAsync(tmp.data(), g->kry_small, (2 * kMaxVec + 1) * sizeof(double),
                          cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  for (int i = 0; i < j1; ++i) h_host[i] = tmp[i] + tmp[kMaxVec + i];
  *wnorm = std::sqrt(std::max(tmp[2 * kMaxVec], 0.0));
  return FV_OK;
}

// cgs2 against a float-float basis (w stays a double vector)
static fv_status cgs2_ffb(const fv_grid* g, const float2* Vf, int j1, double* w, double* h_host,
                          double* wnorm) {
  double* dh1 = g->kry_small;
  double* dh2 = g->kry_small + kMaxVec;
  double* dnn = g->kry_small + 2 * kMaxVec;
  FV_TRY(ffb_dots(g, Vf, j1, w, dh1));
  FV_TRY(ffb_update(g, w, Vf, j1, dh1, -1.0));
  FV_TRY(ffb_dots(g, Vf, j1, w, dh2));
  FV_TRY(ffb_update(g, w, Vf, j1, dh2, -1.0));
  FV_TRY(vec_dots(g, w, g->nvel, 1, w, dnn, true));
  std::vector<double> tmp(2 * kMaxVec + 1);
  FV_CUDA(cudaMemcpyAsync(tmp.data(), g->kry_small, (2 * kMaxVec + 1) * sizeof(double),
                          cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  for (int i = 0; i < j1; ++i) h_host[i] = tmp[i] + tmp[kMaxVec + i];
  *wnorm = std::sqrt(std::max(tmp[2 * kMaxVec], 0.0));
  return FV_OK;
}

// CGS2 of w against the first j1 basis vectors (float-float basis Vf, or the
// FP64 basis V), the coefficients and the norm written into column `Hcol` of
// the device Hessenberg (leading dimension ld) by k_gs_finish, *dscale =
// 1 / norm: nothing returns to the host
static fv_status cgs2_dev(const fv_grid* g, const float2* Vf, const double* V, int j1, double* w,
                          double* Hcol, int ld, double* dscale, bool sub_only) {
  double* dh1 = g->kry_small;
  double* dh2 = g->kry_small + kMaxVec;
  double* dnn = g->kry_small + 2 * kMaxVec;
  if (Vf) {
    FV_TRY(ffb_dots(g, Vf, j1, w, dh1));
    FV_TRY(ffb_update(g, w, Vf, j1, dh1, -1.0));
    FV_TRY(ffb_dots(g, Vf, j1, w, dh2));
    FV_TRY(ffb_update(g, w, Vf, j1, dh2, -1.0));
    FV_TRY(vec_dots(g, w, g->nvel, 1, w, dnn, true));
  } else {
    FV_TRY(vec_dots(g, V, g->nvel, j1, w, dh1, false));
    FV_TRY(vec_update(g, w, V, g->nvel, j1, dh1, -1.0, false));
    FV_TRY(vec_dots(g, V, g->nvel, j1, w, dh2, false));
    FV_TRY(vec_update(g, w, V, g->nvel, j1, dh2, -1.0, false));
    FV_TRY(vec_dots(g, w, g->nvel, 1, w, dnn, false));
  }
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    k_gs_finish<<<1, 128, 0, g->stream>>>(dh1, dh2, dnn, j1, Hcol, ld, dscale, sub_only ? 1 : 0);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

// store w / norm (device scale) as basis column `col`
static fv_status store_scaled(const fv_grid* g, const double* w, const double* dscale, float2* colf,
                              double* cold) {
  {
    LaunchScope ls_(g, FV_K_VECTOR);
    if (colf)
      k_store_ff_dev<<<grid1d(g->nvel), 256, 0, g->stream>>>(g->nvel, w, dscale, colf);
    else
      k_scale_dev<<<grid1d(g->nvel), 256, 0, g->stream>>>(g->nvel, w, dscale, 1, cold);
  }
  FV_CHECK_LAUNCH();
  return FV_OK;
}

static fv_status dot_host(const fv_grid* g, const double* a, const double* b, double* out) {
  double* d = g->kry_small ? g->kry_small + 2 * kMaxVec + 4 : g->d_scal + S_RED;
  FV_TRY(vec_dots(g, a, g->nvel, 1, b, d));
  FV_CUDA(cudaMemcpyAsync(g->h_scal + S_RED, d, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  *out = g->h_scal[S_RED];
  return FV_OK;
}

// W-inner products of nvec columns of V (stride ldv) with w, to the host in
// one synchronisation (FP64)
static fv_status dots_host(const fv_grid* g, const double* V, int64_t ldv, int nvec,
                           const double* w, double* out) {
  double* d = g->kry_small + 3 * kMaxVec;
  FV_TRY(vec_dots(g, V, ldv, nvec, w, d));
  FV_CUDA(cudaMemcpyAsync(out, d, nvec * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  return FV_OK;
}

static fv_status maxabs_host(const fv_grid* g, int64_t n, const double* x, double* out, bool* nan) {
  FV_TRY(reset_scalars(g));
  FV_TRY(vec_maxabs(g, n, x, g->d_scal + S_RED + 1));
  double h[kScalars];
  FV_TRY(fetch_scalars(g, h));
  *out = h[S_RED + 1];
  if (nan) *nan = h[S_NAN] != 0.0;
  return FV_OK;
}

// BiCGstab(2) (Sleijpen & Fokkema 1993) for A_sigma x = b in the W-inner
// product, from x (in/out), shadow residual = the initial residual; the
// BiCGstab(l) recurrences written out for l = 2.  Section 3 runs it from the
// last approximation of a saturated GMRES(m).  Uses Krylov columns 0..7 of
// g->kry as r~, r_0..r_2, u_0..u_2 and the iterate of smallest residual
// (0..9 with a preconditioner: the preconditioned iterate y and M^-1 v).
// Stops when the recursive residual W-norm is <= stop, after max_mv
// products, on a zero BiCG / MR denominator, or when the residual turns
// non-finite or grows 1e6-fold over the smallest seen; x is then the
// iterate of smallest recursive residual.  *mv: products done.
// pre: right preconditioning by the Stokes-type M^-1 (precond_sigma psig):
// the recurrences run on A M^-1 from y = 0 and x becomes x_0 + M^-1 y_best
// at the end (one more preconditioner application, no product).
static fv_status bicgstab2(fv_grid* g, const double* U, const double* b, double* x, double stop,
                           int max_mv, int prec, double sigma, double eps, bool pre, double psig,
                           double tau, int* mv, double* rnorm_out) {
  const int64_t nv = g->nvel;
  double* rt = g->kry;
  double* r[3] = {g->kry + nv, g->kry + 2 * nv, g->kry + 3 * nv};
  double* u[3] = {g->kry + 4 * nv, g->kry + 5 * nv, g->kry + 6 * nv};
  double* xbest = g->kry + 7 * nv;
  double* yit = g->kry + 8 * nv;             // preconditioned iterate
  double* tz = g->kry + 9 * nv;              // M^-1 of the vector being applied
  auto plain = [&](const double* in, double* out) -> fv_status {   // out = (A - tau I) in
    ++*mv;
    FV_TRY(krylov_apply(g, U, in, out, nullptr, sigma, prec, eps, 200, 1.0, nullptr));
    if (tau != 0.0) FV_TRY(vec_axpby(g, nv, 1.0, out, -tau, in, out));
    return FV_OK;
  };
  auto apply = [&](const double* in, double* out) -> fv_status {
    if (pre) {
      FV_TRY(stokes_precond_apply(g, in, tz, psig));
      in = tz;
    }
    return plain(in, out);
  };
  *mv = 0;
  FV_TRY(plain(x, r[0]));
  FV_TRY(vec_axpby(g, nv, -1.0, r[0], 1.0, b, r[0]));
  double* const x0 = x;
  if (pre) {                                 // iterate on y, x = x_0 + M^-1 y
    FV_CUDA(cudaMemsetAsync(yit, 0, nv * sizeof(double), g->stream));
    x = yit;
  }
  FV_CUDA(cudaMemcpyAsync(rt, r[0], nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  FV_CUDA(cudaMemsetAsync(u[0], 0, nv * sizeof(double), g->stream));
  double rho0 = 1.0, alpha = 0.0, omega = 1.0, rr, rho_next;
  // (r~, r_0) and (r_0, r_0) in one pass: r~ and r_0 are adjacent columns
  double d2[3];
  FV_TRY(dots_host(g, rt, nv, 2, r[0], d2));
  rho_next = d2[0];
  rr = d2[1];
  double rnorm = std::sqrt(rr), best = rnorm;
  FV_CUDA(cudaMemcpyAsync(xbest, x, nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  auto finish = [&]() -> fv_status {        // hand back the best iterate
    FV_TRY(check_products(g, prec));
    if (pre) {
      FV_TRY(stokes_precond_apply(g, xbest, tz, psig));
      FV_TRY(vec_axpby(g, nv, 1.0, x0, 1.0, tz, x0));
    } else {
      FV_CUDA(cudaMemcpyAsync(x, xbest, nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    }
    *rnorm_out = best;
    return FV_OK;
  };
  while (rnorm > stop && *mv + 4 <= max_mv) {
    rho0 = -omega * rho0;
    // BiCG part: two steps, each raising the degree of the kept powers by one
    for (int j = 0; j < 2; ++j) {
      double rho1, gam;
      if (j == 0) rho1 = rho_next;                 // from the end of the previous cycle
      else FV_TRY(dot_host(g, r[j], rt, &rho1));
      if (rho0 == 0.0 || !std::isfinite(rho1)) return finish();
      const double beta = alpha * rho1 / rho0;
      rho0 = rho1;
      for (int i = 0; i <= j; ++i) FV_TRY(vec_axpby(g, nv, 1.0, r[i], -beta, u[i], u[i]));
      FV_TRY(apply(u[j], u[j + 1]));
      FV_TRY(dot_host(g, u[j + 1], rt, &gam));
      if (gam == 0.0 || !std::isfinite(gam)) return finish();
      alpha = rho0 / gam;
      for (int i = 0; i <= j; ++i) FV_TRY(vec_axpby(g, nv, 1.0, r[i], -alpha, u[i + 1], r[i]));
      FV_TRY(apply(r[j], r[j + 1]));
      FV_TRY(vec_axpby(g, nv, 1.0, x, alpha, u[0], x));
    }
    // MR part: orthogonalise r_2 against r_1, then the minimal-residual
    // polynomial of degree 2 (gamma', gamma, gamma'' of the l = 2 case)
    // (r_0, r_1), (r_1, r_1), (r_2, r_1) in one pass (r_0..r_2 are adjacent
    // columns), then (r_0, r_2), (r_2, r_2) after r_2 is orthogonalised
    double d3[3];
    FV_TRY(dots_host(g, r[0], nv, 3, r[1], d3));
    const double c01 = d3[0], s1 = d3[1], c12 = d3[2];
    if (!(s1 > 0.0) || !std::isfinite(s1)) return finish();
    const double gp1 = c01 / s1;
    const double tau12 = c12 / s1;
    FV_TRY(vec_axpby(g, nv, 1.0, r[2], -tau12, r[1], r[2]));
    FV_TRY(dots_host(g, r[0], 2 * nv, 2, r[2], d2));
    const double c02 = d2[0], s2 = d2[1];
    if (!(s2 > 0.0) || !std::isfinite(s2)) return finish();
    const double gp2 = c02 / s2;
    const double g2 = gp2, g1 = gp1 - tau12 * g2, gpp1 = g2;
    omega = g2;
    FV_TRY(vec_axpby(g, nv, 1.0, x, g1, r[0], x));
    FV_TRY(vec_axpby(g, nv, 1.0, x, gpp1, r[1], x));
    FV_TRY(vec_axpby(g, nv, 1.0, r[0], -gp2, r[2], r[0]));
    FV_TRY(vec_axpby(g, nv, 1.0, r[0], -gp1, r[1], r[0]));
    FV_TRY(vec_axpby(g, nv, 1.0, u[0], -g2, u[2], u[0]));
    FV_TRY(vec_axpby(g, nv, 1.0, u[0], -g1, u[1], u[0]));
    FV_TRY(dots_host(g, rt, nv, 2, r[0], d2));
    FV_TRY(check_products(g, prec));
    rho_next = d2[0];
    rr = d2[1];
    rnorm = std::sqrt(rr);
    if (!std::isfinite(rnorm) || rnorm > 1e6 * best) return finish();
    if (rnorm < best) {
      best = rnorm;
      FV_CUDA(cudaMemcpyAsync(xbest, x, nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
    }
  }
  return finish();
}

}  // namespace fv

using namespace fv;

static fv_status check_grid(const fv_grid* g, const char* who) {
  if (!g) { set_error(std::string(who) + ": grid is NULL"); return FV_EINVAL; }
  return FV_OK;
}

extern "C" {

fv_status ns_residual(const fv_grid* g, const double* U, const double* P, double* F_mom,
                      double* F_div) {
  FV_TRY(check_grid(g, "ns_residual"));
  if (!U || !P || !F_mom || !F_div) { set_error("ns_residual: NULL pointer"); return FV_EINVAL; }
  return launch_residual(g, U, P, F_mom, F_div);
}

fv_status ns_jacvec(const fv_grid* g, const double* U, const double* v, double* Jv, int prec) {
  FV_TRY(check_grid(g, "ns_jacvec"));
  if (!U || !v || !Jv) { set_error("ns_jacvec: NULL pointer"); return FV_EINVAL; }
  if (prec != FV_FP64 && prec != FV_MIXED && prec != FV_FF) { set_error("ns_jacvec: bad prec"); return FV_EINVAL; }
  if (v == Jv || U == Jv) { set_error("ns_jacvec: output aliases an input"); return FV_EINVAL; }
  if (prec == FV_FF) return launch_jv_ff_out64(g, U, v, Jv, 0.0);
  return launch_momentum_jac(g, U, v, Jv, prec, 0.0);
}

fv_status fv_dot_w(const fv_grid* g, const double* a, const double* b, double* out) {
  FV_TRY(check_grid(g, "fv_dot_w"));
  if (!a || !b || !out) { set_error("fv_dot_w: NULL pointer"); return FV_EINVAL; }
  return dot_host(g, a, b, out);
}

fv_status simple_krylov_solve(const fv_grid* g, const double* U, const double* v_in, double* v_out,
                              double* p_out, const fv_simple_opts* opts, fv_simple_stats* stats) {
  FV_TRY(check_grid(g, "simple_krylov_solve"));
  if (!v_in || !v_out) { set_error("simple_krylov_solve: NULL pointer"); return FV_EINVAL; }
  if (!U && !g->base_ptr) {
    set_error("simple_krylov_solve: U is NULL and no base flow is registered (fv_grid_set_base)");
    return FV_EINVAL;
  }
  if (v_in == v_out) { set_error("simple_krylov_solve: v_in and v_out alias"); return FV_EINVAL; }
  fv_simple_opts o = {};
  if (opts) o = *opts;
  if (o.eps <= 0.0) o.eps = 1e-8;
  if (o.max_pass <= 0) o.max_pass = 200;
  if (o.omega <= 0.0) o.omega = 1.0;
  if (o.omega > 1.0 || (o.prec != FV_FP64 && o.prec != FV_MIXED && o.prec != FV_FF) || o.sigma < 0.0) {
    set_error("simple_krylov_solve: bad option");
    return FV_EINVAL;
  }
  if (o.pressure < 0 || o.pressure > 1 || (o.pressure == 1 && o.prec != FV_FP64) ||
      o.pressure_rtol < 0.0 || o.pressure_rtol >= 1.0) {
    set_error("simple_krylov_solve: bad option (pressure 1 needs FV_FP64, 0 <= pressure_rtol < 1)");
    return FV_EINVAL;
  }
  SimpleResult r;
  fv_status s;
  if (o.pressure == 1) {                       // FP64 loop with multigrid pressure solves
    fv_mg_opts mo = {};
    mo.rtol = o.pressure_rtol > 0.0 ? o.pressure_rtol : 1e-3;
    mo.max_iter = 100;
    mo.nu = 1;
    mo.omega = 1.0;
    FV_TRY(launch_momentum_jac(g, U ? U : g->base_ptr, v_in, v_out, FV_FP64, o.sigma));
    s = simple_loop(g, v_out, g->vel_buf[0], v_out, p_out, o.eps, o.max_pass, FV_FP64, o.omega, &r,
                    0.0, &mo);
    if (s == FV_OK && o.sigma != 0.0) FV_TRY(vec_axpby(g, g->nvel, 1.0, v_out, -o.sigma, v_in, v_out));
    if (stats) {
      stats->passes = r.passes;
      stats->phi_first = r.phi_first;
      stats->phi_last = r.phi_last;
      stats->div_max = r.div_max;
    }
    return s;
  }
  const bool no_sync = o.async != 0 && o.prec != FV_FP64;
  s = krylov_apply(g, U, v_in, v_out, p_out, o.sigma, o.prec, o.eps, o.max_pass, o.omega,
                   no_sync ? nullptr : &r);
  if (stats && !no_sync) {
    stats->passes = r.passes;
    stats->phi_first = r.phi_first;
    stats->phi_last = r.phi_last;
    stats->div_max = r.div_max;
  }
  return s;
}

fv_status simple_krylov_solve_guess(const fv_grid* g, fv_unet* u, const double* U,
                                    const double* v_in, double* v_out, double* p_out,
                                    const fv_simple_opts* opts, fv_simple_stats* stats) {
  FV_TRY(check_grid(g, "simple_krylov_solve_guess"));
  if (!u || !U || !v_in || !v_out) { set_error("simple_krylov_solve_guess: NULL pointer"); return FV_EINVAL; }
  if (v_in == v_out) { set_error("simple_krylov_solve_guess: v_in and v_out alias"); return FV_EINVAL; }
  fv_simple_opts o = {};
  if (opts) o = *opts;
  if (o.eps <= 0.0) o.eps = 1e-8;
  if (o.max_pass <= 0) o.max_pass = 200;
  if (o.omega <= 0.0) o.omega = 1.0;
  if (o.omega > 1.0 || (o.prec != FV_MIXED && o.prec != FV_FF) || o.sigma < 0.0 || o.max_pass < 2) {
    set_error("simple_krylov_solve_guess: bad option (prec FV_MIXED or FV_FF, max_pass >= 2)");
    return FV_EINVAL;
  }
  SimpleResult r;
  fv_status s;
  if (o.prec == FV_FF) {
    FV_TRY(launch_jv_ff(g, U, v_in, g->vff[1], o.sigma));
    FV_TRY(launch_div_ff(g, g->vff[1], g->r32));
    FV_TRY(unet_guess_f32(u, g, g->r32, g->phi32));
    s = simple_loop_ff(g, v_out, p_out, v_in, o.sigma, o.eps, o.max_pass, o.omega, &r, true, g->phi32);
  } else {
    FV_TRY(launch_jv_f32(g, U, v_in, g->w32, o.sigma));
    FV_TRY(launch_div_f32(g, g->w32, g->r32));
    FV_TRY(unet_guess_f32(u, g, g->r32, g->phi32));
    s = simple_loop_ff(g, v_out, p_out, v_in, o.sigma, o.eps, o.max_pass, o.omega, &r, false, g->phi32);
  }
  if (stats) {
    stats->passes = r.passes;
    stats->phi_first = r.phi_first;
    stats->phi_last = r.phi_last;
    stats->div_max = r.div_max;
  }
  if (s == FV_OK) FV_CUDA(cudaStreamSynchronize(g->stream));
  return s;
}

fv_status ns_divergence(const fv_grid* g, const double* v, double* r) {
  FV_TRY(check_grid(g, "ns_divergence"));
  if (!v || !r) { set_error("ns_divergence: NULL pointer"); return FV_EINVAL; }
  return launch_divergence(g, v, r, nullptr);
}

// ---------------------------------------------------------------- Newton --
fv_status newton_steady(fv_grid* g, double* U, double* P, const fv_newton_opts* opts,
                        fv_newton_stats* stats) {
  FV_TRY(check_grid(g, "newton_steady"));
  if (!U || !P) { set_error("newton_steady: NULL pointer"); return FV_EINVAL; }
  fv_newton_opts o = {};
  if (opts) o = *opts;
  if (o.tol <= 0) o.tol = 1e-10;
  if (o.max_newton <= 0) o.max_newton = 30;
  if (o.gmres_m <= 0) o.gmres_m = 100;
  if (o.gmres_max_it <= 0) o.gmres_max_it = 20000;
  if (o.gmres_rtol <= 0) o.gmres_rtol = 1e-8;
  if (o.sigma <= 0) o.sigma = 10.0;
  if (o.simple_eps <= 0) o.simple_eps = 1e-10;
  if (o.gmres_sat <= 0) o.gmres_sat = 0.5;
  if (o.gmres_m > kMaxVec - 2 || (o.prec != FV_FP64 && o.prec != FV_MIXED && o.prec != FV_FF) ||
      o.linear < FV_LIN_GMRES_BICGSTAB || o.linear > FV_LIN_BICGSTAB) {
    set_error("newton_steady: bad option (gmres_m <= 128, prec, linear)");
    return FV_EINVAL;
  }
  if (o.precond < 0 || o.precond > 1 || o.precond_sigma < 0.0 || o.forcing < 0 || o.forcing > 1 ||
      !(o.tau >= 0.0)) {
    set_error("newton_steady: bad option (precond 0 or 1, precond_sigma >= 0, forcing 0 or 1, tau >= 0)");
    return FV_EINVAL;
  }
  const bool pre = o.precond == 1;            // flexible GMRES(m) with the stored M^-1 v_j
  const int m = o.gmres_m;
  const int naug_max = pre ? o.gmres_aug : 0;  // augmentation vectors of the flexible cycles
  if (o.gmres_aug < 0 || o.gmres_aug > 4 || (o.gmres_aug > 0 && (!pre || o.gmres_aug >= m))) {
    set_error("newton_steady: bad option (gmres_aug in [0, 4], < gmres_m, needs precond = 1)");
    return FV_EINVAL;
  }
  FV_TRY(ensure_krylov(g, pre ? std::max(2 * m + 1 + naug_max + 1, 10) : std::max(m + 1, 8)));
  {
    int w;                                     // forget statuses of earlier evaluations
    FV_TRY(graph_take_status(g, &w, false));
  }
  const int64_t nv = g->nvel;
  double* V = g->kry;
  double* Z = pre ? g->kry + (int64_t)(m + 1) * nv : nullptr;   // preconditioned directions
  // the corrections of the latest restart cycles (unit W-norm), the newest
  // in aug[(aug_head - 1) mod (naug_max + 1)]; one slot more holds the
  // correction being formed
  double* aug = pre ? g->kry + (int64_t)(2 * m + 1) * nv : nullptr;
  double* Fm = g->vel_buf[1];
  double* du = g->vel_buf[2];
  fv_newton_stats st = {};
  SimpleResult sr;
  // W-norm floor that keeps the max-norm residual well below tol
  double wmin = 1e300;
  for (int d = 0; d < 3; ++d)
    for (double x : g->h_dx[d]) wmin = std::min(wmin, x);
  const double atol = 1e-3 * o.tol * std::sqrt(0.5 * wmin * wmin * wmin);

  // FV_MIXED: float32 Krylov vectors while they still cut ||F|| by 10x per
  // step, then float64 (the inexact Jacobian of the mixed form limits the
  // linear rate of Newton near the root); the residual is always float64
  int cur_prec = o.prec;
  double prev_res = -1.0, eta_prev = 0.1;
  // errors inside the iteration still report the steps taken
#define NT_TRY(x)                                   \
  do {                                              \
    const fv_status s_ = (x);                       \
    if (s_ != FV_OK) {                              \
      if (stats) *stats = st;                       \
      return s_;                                    \
    }                                               \
  } while (0)
#define NT_CUDA(x)                                                       \
  do {                                                                   \
    const cudaError_t e_ = (x);                                          \
    if (e_ != cudaSuccess) NT_TRY(::fv::cuda_fail(e_, #x, __FILE__, __LINE__)); \
  } while (0)
  for (int it = 0; it <= o.max_newton; ++it) {
    // continuity part of the Newton correction: project U
    NT_TRY(launch_zero_walls(g, U));
    NT_TRY(project_inplace(g, U, nullptr, FV_MIXED, 1e-13, &sr));
    // momentum residual with P = 0, projected: F_m = N(U) - G P(U), and
    // P(U) = (D G)^+ D N(U) accumulated by the projection
    NT_CUDA(cudaMemsetAsync(P, 0, g->ncell * sizeof(double), g->stream));
    NT_TRY(launch_residual(g, U, P, Fm, nullptr));
    NT_TRY(project_inplace(g, Fm, P, FV_MIXED, 1e-13, &sr));
    double fmax, dmax;
    bool nan1 = false, nan2 = false;
    NT_TRY(maxabs_host(g, nv, Fm, &fmax, &nan1));
    NT_TRY(launch_divergence(g, U, g->cell_buf[2], nullptr));
    NT_TRY(maxabs_host(g, g->ncell, g->cell_buf[2], &dmax, &nan2));
    const double res = std::max(fmax, dmax);
    if (it < 64) st.res_hist[it] = res;
    st.res_final = res;
    st.iterations = it;
    if (nan1 || nan2 || !std::isfinite(res)) {
      if (stats) *stats = st;
      set_error("newton_steady: NaN in the residual");
      return FV_ENAN;
    }
    if (res < o.tol) {
      if (stats) *stats = st;
      return FV_OK;
    }
    if (it == o.max_newton) break;
    if (cur_prec == FV_MIXED && prev_res > 0.0 && res > 0.1 * prev_res) cur_prec = FV_FP64;
    // relative tolerance of this correction: fixed, or the Eisenstat-Walker
    // forcing term (their choice 2: gamma 0.9, exponent 2, with its safeguard)
    double eta = o.gmres_rtol;
    if (o.forcing == 1) {
      double e = 0.1;
      if (prev_res > 0.0) {
        const double q = res / prev_res;
        e = 0.9 * q * q;
        const double safe = 0.9 * eta_prev * eta_prev;
        if (safe > 0.1) e = std::max(e, safe);
      }
      eta = std::min(0.1, std::max(e, o.gmres_rtol));
      eta_prev = eta;
    }
    prev_res = res;
    const double lin_rtol = cur_prec == FV_MIXED ? std::max(eta, 1e-6) : eta;
    // the Jacobian of this step: U converted once for all its Krylov vectors
    NT_TRY(set_base(g, U));

    // GMRES(m) for A_sigma du = Fm, du = 0 initially
    NT_CUDA(cudaMemsetAsync(du, 0, nv * sizeof(double), g->stream));
    double bnorm;
    NT_TRY(dot_host(g, Fm, Fm, &bnorm));
    bnorm = std::sqrt(bnorm);
    const double stop = std::max(lin_rtol * bnorm, atol);
    int its = 0;
    bool first = true, converged = false;
    double prev_beta = bnorm;
    double lin_res = bnorm;                    // latest residual estimate of this correction
    int naug = 0, aug_head = 0;                // augmentation vectors of this solve
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), hcol(m + 2);
    while (o.linear != FV_LIN_BICGSTAB) {
      // r = b - A du
      if (first) {
        NT_CUDA(cudaMemcpyAsync(V, Fm, nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
      } else {
        NT_TRY(krylov_apply(g, nullptr, du, V, nullptr, o.sigma, cur_prec, o.simple_eps, 200, 1.0,
                            nullptr));
        if (o.tau != 0.0) NT_TRY(vec_axpby(g, nv, 1.0, V, -o.tau, du, V));
        NT_TRY(vec_axpby(g, nv, -1.0, V, 1.0, Fm, V));
      }
      first = false;
      double beta;
      NT_TRY(dot_host(g, V, V, &beta));
      beta = std::sqrt(beta);
      lin_res = beta;
      if (beta <= stop) { converged = true; break; }
      if (its >= o.gmres_max_it) break;
      // saturated: the last restart cycle cut the residual by less than gmres_sat
      if (o.linear == FV_LIN_GMRES_BICGSTAB && its > 0 && beta > o.gmres_sat * prev_beta) break;
      prev_beta = beta;
      NT_TRY(vec_axpby(g, nv, 1.0 / beta, V, 0.0, nullptr, V));
      std::fill(gv.begin(), gv.end(), 0.0);
      gv[0] = beta;
      int jdone = 0;
      for (int j = 0; j < m; ++j) {
        double* w = V + (int64_t)(j + 1) * nv;
        const double* vj = V + (int64_t)j * nv;
        if (pre) {                             // z_j = M^-1 v_j, w = A z_j
          double* zj = Z + (int64_t)j * nv;
          const int ja = j - (m - naug);           // the last naug steps take earlier corrections
          if (ja >= 0) {
            const int slot = ((aug_head - 1 - ja) % (naug_max + 1) + (naug_max + 1)) % (naug_max + 1);
            NT_CUDA(cudaMemcpyAsync(zj, aug + (int64_t)slot * nv, nv * sizeof(double),
                                    cudaMemcpyDeviceToDevice, g->stream));
          } else {
            NT_TRY(stokes_precond_apply(g, vj, zj, o.precond_sigma));
          }
          vj = zj;
        }
        NT_TRY(krylov_apply(g, nullptr, vj, w, nullptr, o.sigma, cur_prec, o.simple_eps,
                            200, 1.0, nullptr));
        if (o.tau != 0.0) NT_TRY(vec_axpby(g, nv, 1.0, w, -o.tau, vj, w));
        double hn;
        NT_TRY(cgs2(g, V, j + 1, w, hcol.data(), &hn, cur_prec != FV_FP64));
        if (hn > 0) NT_TRY(vec_axpby(g, nv, 1.0 / hn, w, 0.0, nullptr, w));
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hcol[i];
        H[(size_t)(j + 1) * m + j] = hn;
        for (int i = 0; i < j; ++i) {
          const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
        }
        const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
        const double den = std::hypot(a, b);
        cs[j] = den == 0 ? 1.0 : a / den;
        sn[j] = den == 0 ? 0.0 : b / den;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        gv[j + 1] = -sn[j] * gv[j];
        gv[j] = cs[j] * gv[j];
        ++its;
        jdone = j + 1;
        if (std::fabs(gv[j + 1]) <= stop || its >= o.gmres_max_it || hn == 0) break;
      }
      NT_TRY(check_products(g, cur_prec));
      // y = R^{-1} g ; du += V y
      std::vector<double> y(jdone);
      for (int i = jdone - 1; i >= 0; --i) {
        double s = gv[i];
        for (int k = i + 1; k < jdone; ++k) s -= H[(size_t)i * m + k] * y[k];
        y[i] = s / H[(size_t)i * m + i];
      }
      NT_CUDA(cudaMemcpyAsync(g->kry_small, y.data(), jdone * sizeof(double), cudaMemcpyHostToDevice,
                              g->stream));
      if (naug_max > 0) {
        // this cycle's correction Z y, kept (normalised) for the next cycles
        double* dc = aug + (int64_t)aug_head * nv;
        NT_CUDA(cudaMemsetAsync(dc, 0, nv * sizeof(double), g->stream));
        NT_TRY(vec_update(g, dc, Z, nv, jdone, g->kry_small, 1.0, cur_prec != FV_FP64));
        NT_TRY(vec_axpby(g, nv, 1.0, du, 1.0, dc, du));
        double dn;
        NT_TRY(dot_host(g, dc, dc, &dn));
        dn = std::sqrt(dn);
        if (dn > 0.0 && std::isfinite(dn)) {
          NT_TRY(vec_axpby(g, nv, 1.0 / dn, dc, 0.0, nullptr, dc));
          aug_head = (aug_head + 1) % (naug_max + 1);
          naug = std::min(naug + 1, naug_max);
        }
      } else {
        NT_TRY(vec_update(g, du, pre ? Z : V, nv, jdone, g->kry_small, 1.0, cur_prec != FV_FP64));
      }
      NT_CUDA(cudaStreamSynchronize(g->stream));
      lin_res = std::fabs(gv[jdone]);
    }
    st.gmres_total += its;
    if (!converged && o.linear != FV_LIN_GMRES && its < o.gmres_max_it) {
      // BiCGstab(2) from the last approximation; after a breakdown it starts
      // again from its best iterate (new shadow residual) while the product
      // budget lasts and each start cuts the residual by 10 % or more
      int budget = o.gmres_max_it - its;
      double prev = HUGE_VAL;
      for (int rs = 0; rs < 64 && budget > 4; ++rs) {
        int mv = 0;
        double rn;
        NT_TRY(bicgstab2(g, nullptr, Fm, du, stop, budget, cur_prec, o.sigma, o.simple_eps, pre,
                         o.precond_sigma, o.tau, &mv, &rn));
        st.bicgstab_total += mv;
        budget -= mv;
        lin_res = std::min(lin_res, rn);
        if (rn <= stop || !(rn < 0.9 * prev)) break;
        prev = rn;
      }
    }
    if (it < 64) st.lin_hist[it] = bnorm > 0.0 ? lin_res / bnorm : 0.0;
    NT_TRY(vec_axpby(g, nv, 1.0, U, -1.0, du, U));
  }
#undef NT_TRY
#undef NT_CUDA
  if (stats) *stats = st;
  set_error("newton_steady: no convergence within max_newton");
  return FV_ENOCONV;
}

// --------------------------------------------------------------- Arnoldi --
fv_status arnoldi_leading(const fv_grid* gc, const double* U, const double* v0, int m, int nev,
                          double* lam_re, double* lam_im, double* evec,
                          const fv_arnoldi_opts* opts, fv_arnoldi_stats* stats) {
  fv_grid* g = const_cast<fv_grid*>(gc);
  FV_TRY(check_grid(g, "arnoldi_leading"));
  if (!U || !v0 || !lam_re || !lam_im) { set_error("arnoldi_leading: NULL pointer"); return FV_EINVAL; }
  if (nev < 1 || nev > 64 || m < nev + 2 || m > 128) {
    set_error("arnoldi_leading: need 1 <= nev <= 64 and nev + 2 <= m <= 128");
    return FV_EINVAL;
  }
  fv_arnoldi_opts o = {};
  if (opts) o = *opts;
  if (o.tol <= 0) o.tol = 1e-10;
  if (o.max_restarts <= 0) o.max_restarts = 5000;
  if (o.sigma <= 0) o.sigma = 10.0;
  if (o.simple_eps <= 0) o.simple_eps = 1e-10;
  if (o.prec != FV_FP64 && o.prec != FV_MIXED && o.prec != FV_FF) { set_error("arnoldi_leading: bad prec"); return FV_EINVAL; }
  // the basis of the mixed and float-float forms is stored as float-float
  // pairs and orthogonalised and recombined in float-float arithmetic (FP32
  // pipes): columns 0..m, then two double columns for the operand and the
  // new vector; the FP64 form keeps an FP64 basis
  const bool gs_ff = o.prec != FV_FP64;
  FV_TRY(ensure_krylov(g, gs_ff ? m + 3 : m + 1));
  {
    int w;                                     // forget statuses of earlier evaluations
    FV_TRY(graph_take_status(g, &w, false));
  }
  FV_TRY(set_base(g, U));                      // U converted once for every Krylov vector
  const int64_t nv = g->nvel;
  double* V = g->kry;
  float2* Vf = (float2*)g->kry;
  double* xs = g->kry + (int64_t)(m + 1) * nv;
  double* ws = xs + nv;
  SimpleResult sr;
  // v_0 = P x_0 / ||P x_0||
  double* x0 = gs_ff ? xs : V;
  FV_CUDA(cudaMemcpyAsync(x0, v0, nv * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  FV_TRY(launch_zero_walls(g, x0));
  FV_TRY(project_inplace(g, x0, nullptr, FV_MIXED, 1e-13, &sr));
  double nrm;
  FV_TRY(dot_host(g, x0, x0, &nrm));
  if (!(nrm > 0)) { set_error("arnoldi_leading: start vector has no solenoidal part"); return FV_EINVAL; }
  if (gs_ff)
    FV_TRY(ffb_store(g, x0, 1.0 / std::sqrt(nrm), Vf));
  else
    FV_TRY(vec_axpby(g, nv, 1.0 / std::sqrt(nrm), V, 0.0, nullptr, V));

  // The Arnoldi steps of a cycle run without host round trips: each
  // Gram-Schmidt writes its coefficients and the new vector's norm into the
  // FP64 Hessenberg H held in device memory, and the new basis vector is
  // scaled by that norm on the device.  The host copies H once per cycle for
  // the small dense work (Ritz values by Francis QR, Ritz estimates, exact
  // shifts, the recombination matrix; fv_dense.cu) and sends the
  // recombination matrix back.
  if (!g->d_arn) {
    const size_t bytes = (size_t)((kMaxVec + 1) * kMaxVec + 8) * sizeof(double);
    cudaError_t e = cudaMalloc(&g->d_arn, bytes);
    if (e != cudaSuccess) {
      (void)cudaGetLastError();
      g->d_arn = nullptr;
      set_error("arnoldi_leading: device area allocation failed");
      return FV_ENOMEM;
    }
  }
  double* dH = (double*)g->d_arn;
  double* dsc = dH + (kMaxVec + 1) * kMaxVec;   // 1 / norm of the new vector
  FV_CUDA(cudaMemsetAsync(dH, 0, (size_t)(m + 1) * m * sizeof(double), g->stream));
  std::vector<double> H((size_t)(m + 1) * m, 0.0);
  std::vector<double> Hm((size_t)m * m), Q((size_t)m * m), wr(m), wi(m);
  const int k_base = std::min(nev + (m - nev) / 2, m - 2);
  int k = 0, matvecs = 0;
  const double eps23 = std::pow(2.2204460492503131e-16, 2.0 / 3.0);
  for (int restart = 0; restart < o.max_restarts; ++restart) {
    for (int j = k; j < m; ++j) {
      const double* xj = V + (int64_t)j * nv;
      double* w = V + (int64_t)(j + 1) * nv;
      if (gs_ff) {
        FV_TRY(ffb_load(g, Vf + (int64_t)j * nv, xs));
        xj = xs;
        w = ws;
      }
      FV_TRY(krylov_apply(g, nullptr, xj, w, nullptr, o.sigma, o.prec, o.simple_eps, 200, 1.0, nullptr));
      ++matvecs;
      FV_TRY(cgs2_dev(g, gs_ff ? Vf : nullptr, V, j + 1, w, dH + j, m, dsc, false));
      FV_TRY(store_scaled(g, w, dsc, gs_ff ? Vf + (int64_t)(j + 1) * nv : nullptr, w));
    }
    FV_TRY(check_products(g, o.prec));
    FV_CUDA(cudaMemcpyAsync(H.data(), dH, (size_t)(m + 1) * m * sizeof(double), cudaMemcpyDeviceToHost,
                            g->stream));
    FV_CUDA(cudaStreamSynchronize(g->stream));
    for (int j = k; j < m; ++j) {
      const double hn = H[(size_t)(j + 1) * m + j];
      if (!(hn > 0) || !std::isfinite(hn)) { set_error("arnoldi_leading: breakdown"); return FV_ENAN; }
    }
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) Hm[(size_t)i * m + j] = H[(size_t)i * m + j];
    if (!hess_eigenvalues(m, Hm.data(), wr.data(), wi.data())) {
      set_error("arnoldi_leading: Hessenberg QR did not converge");
      return FV_ENOCONV;
    }
    std::vector<int> ord(m);
    for (int i = 0; i < m; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) {
      if (wr[a] != wr[b]) return wr[a] > wr[b];
      return wi[a] > wi[b];
    });
    const double fnorm = std::fabs(H[(size_t)m * m + (m - 1)]);
    std::vector<double> resid(nev), yr(m), yi(m);
    int nconv = 0;
    for (int q = 0; q < nev; ++q) {
      const int id = ord[q];
      hess_eigvec(m, Hm.data(), wr[id], wi[id], yr.data(), yi.data());
      resid[q] = fnorm * std::hypot(yr[m - 1], yi[m - 1]);
      const double sc = std::max(std::hypot(wr[id], wi[id]), eps23);
      if (resid[q] <= o.tol * sc) ++nconv;
    }
    if (nconv >= nev) {
      for (int q = 0; q < nev; ++q) { lam_re[q] = wr[ord[q]]; lam_im[q] = wi[ord[q]]; }
      if (stats) {
        stats->restarts = restart;
        stats->matvecs = matvecs;
        for (int q = 0; q < nev && q < 64; ++q) stats->ritz_resid[q] = resid[q];
      }
      if (evec) {
        // leading Ritz vector x = V y (complex), unit W-norm, phase: its
        // largest-modulus entry real positive, found by a device argmax
        hess_eigvec(m, Hm.data(), wr[ord[0]], wi[ord[0]], yr.data(), yi.data());
        std::vector<double> C((size_t)m * 2);
        for (int i = 0; i < m; ++i) { C[2 * i] = yr[i]; C[2 * i + 1] = yi[i]; }
        FV_CUDA(cudaMemcpyAsync(g->kry_small, C.data(), C.size() * sizeof(double),
                                cudaMemcpyHostToDevice, g->stream));
        if (gs_ff)
          FV_TRY(ffb_combine<double>(g, Vf, m, g->kry_small, 2, evec));
        else
          FV_TRY(vec_combine(g, V, nv, m, g->kry_small, 2, evec, nv, false));
        double a2, b2;
        FV_TRY(dot_host(g, evec, evec, &a2));
        FV_TRY(dot_host(g, evec + nv, evec + nv, &b2));
        const double inv = 1.0 / std::sqrt(a2 + b2);
        const int nb = (int)std::min<int64_t>(152 * 4, (nv + 255) / 256);
        double* pv = (double*)g->d_part;
        int64_t* pidx = (int64_t*)(pv + 1024);
        double* big = pv + 2048;
        {
          LaunchScope ls_(g, FV_K_VECTOR);
          k_absmax_c<<<nb, 256, 0, g->stream>>>(nv, evec, evec + nv, pv, pidx);
          k_absmax_c_final<<<1, 32, 0, g->stream>>>(nb, pv, pidx, evec, evec + nv, big);
        }
        FV_CHECK_LAUNCH();
        double hb[2];
        FV_CUDA(cudaMemcpyAsync(hb, big, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
        FV_CUDA(cudaStreamSynchronize(g->stream));
        const double bm = std::sqrt(hb[0] * hb[0] + hb[1] * hb[1]);
        const double pr = hb[0] / bm, pi = -hb[1] / bm;
        // (a + i b)(pr + i pi) = (a pr - b pi) + i (a pi + b pr)
        const double Cph[4] = {pr * inv, pi * inv, -pi * inv, pr * inv};
        FV_CUDA(cudaMemcpyAsync(g->kry_small, Cph, 4 * sizeof(double), cudaMemcpyHostToDevice, g->stream));
        FV_TRY(vec_combine(g, evec, nv, 2, g->kry_small, 2, evec, nv, gs_ff));
        FV_CUDA(cudaStreamSynchronize(g->stream));
      }
      return FV_OK;
    }
    // implicit restart with the m - k unwanted Ritz values as exact shifts
    k = k_base;
    {
      const int a = ord[k - 1], b = ord[k];
      if (wi[a] != 0.0 && wi[b] == -wi[a] && wr[b] == wr[a]) ++k;
    }
    for (int i = 0; i < m * m; ++i) Q[i] = 0.0;
    for (int i = 0; i < m; ++i) Q[(size_t)i * m + i] = 1.0;
    for (int q = k; q < m; ++q) {
      const int id = ord[q];
      if (wi[id] != 0.0 && q + 1 < m && wi[ord[q + 1]] == -wi[id] && wr[ord[q + 1]] == wr[id]) {
        francis_double_step(m, Hm.data(), Q.data(), wr[id], wi[id]);
        ++q;
      } else {
        single_shift_step(m, Hm.data(), Q.data(), wr[id]);
      }
    }
    // f = V Q e_{k+1} Hs[k][k-1] + f_m Q[m-1][k-1]; new V_k = V Q[:, :k]
    const double fscale = H[(size_t)m * m + (m - 1)] * Q[(size_t)(m - 1) * m + (k - 1)];
    const double bsub = Hm[(size_t)k * m + (k - 1)];
    std::vector<double> C((size_t)(m + 1) * (k + 1), 0.0);
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < k; ++c) C[(size_t)i * (k + 1) + c] = Q[(size_t)i * m + c];
    for (int i = 0; i < m; ++i) C[(size_t)i * (k + 1) + k] = Q[(size_t)i * m + k] * bsub;
    C[(size_t)m * (k + 1) + k] = fscale;
    FV_CUDA(cudaMemcpyAsync(g->kry_small, C.data(), C.size() * sizeof(double),
                            cudaMemcpyHostToDevice, g->stream));
    if (gs_ff) {
      FV_TRY(ffb_combine<float2>(g, Vf, m + 1, g->kry_small, k + 1, Vf));
      FV_TRY(ffb_load(g, Vf + (int64_t)k * nv, ws));
    } else {
      FV_TRY(vec_combine(g, V, nv, m + 1, g->kry_small, k + 1, V, nv, false));
    }
    // the new H: the leading k x k block of the shifted Hm; H[k][k-1] = ||f||
    // after f is re-orthogonalised against the kept vectors (on the device)
    std::fill(H.begin(), H.end(), 0.0);
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) H[(size_t)i * m + j] = Hm[(size_t)i * m + j];
    FV_CUDA(cudaMemcpyAsync(dH, H.data(), (size_t)(m + 1) * m * sizeof(double), cudaMemcpyHostToDevice,
                            g->stream));
    double* f = gs_ff ? ws : V + (int64_t)k * nv;
    FV_TRY(cgs2_dev(g, gs_ff ? Vf : nullptr, V, k, f, dH + (k - 1), m, dsc, true));
    FV_TRY(store_scaled(g, f, dsc, gs_ff ? Vf + (int64_t)k * nv : nullptr, f));
  }
  set_error("arnoldi_leading: max_restarts reached");
  return FV_ENOCONV;
}

// --------------------------------------------------------- critical Re --
fv_status fv_critical_re(fv_grid* g, double* U, double* P, const double* v0, double re0, double re1,
                         const fv_critical_opts* opts, double* re_cr, double* omega_cr,
                         fv_critical_stats* stats) {
  FV_TRY(check_grid(g, "fv_critical_re"));
  if (!U || !P || !v0 || !re_cr || !omega_cr || !(re0 > 0) || !(re1 > 0) || re0 == re1) {
    set_error("fv_critical_re: bad argument");
    return FV_EINVAL;
  }
  fv_critical_opts o = {};
  if (opts) o = *opts;
  if (o.rtol <= 0) o.rtol = 1e-8;
  if (o.max_iter <= 0) o.max_iter = 30;
  if (o.m <= 0) o.m = 30;
  if (o.nev <= 0) o.nev = 4;
  if (o.newton_tol <= 0) o.newton_tol = 1e-10;
  if (o.arnoldi_tol <= 0) o.arnoldi_tol = 1e-10;
  fv_critical_stats st = {};
  fv_newton_opts no = {};
  no.tol = o.newton_tol;
  no.prec = o.prec;
  no.precond = o.precond;
  no.precond_sigma = o.precond_sigma;
  no.forcing = o.forcing;
  no.tau = o.tau;
  no.max_newton = o.max_newton;
  fv_arnoldi_opts ao = {};
  ao.tol = o.arnoldi_tol;
  ao.prec = o.prec;
  ao.max_restarts = o.max_restarts;
  std::vector<double> lr(o.nev), li(o.nev);
  // sigma(Re): Newton from the current U, P, then the leading eigenvalue
  auto sigma = [&](double re, double* s, double* w) -> fv_status {
    FV_TRY(fv_grid_set_re(g, re));
    FV_TRY(newton_steady(g, U, P, &no, nullptr));
    FV_TRY(arnoldi_leading(g, U, v0, o.m, o.nev, lr.data(), li.data(), nullptr, &ao, nullptr));
    *s = lr[0];
    *w = std::fabs(li[0]);
    if (st.evaluations < 64) {
      st.re_hist[st.evaluations] = re;
      st.sigma_hist[st.evaluations] = *s;
      st.omega_hist[st.evaluations] = *w;
    }
    ++st.evaluations;
    return FV_OK;
  };
  double s0, w0, s1, w1;
  fv_status rc = sigma(re0, &s0, &w0);
  if (rc == FV_OK) rc = sigma(re1, &s1, &w1);
  double a = re0, b = re1;
  fv_status out = FV_ENOCONV;
  for (int it = 0; rc == FV_OK && it < o.max_iter; ++it) {
    if (s1 == s0) { set_error("fv_critical_re: flat secant"); out = FV_ENOCONV; break; }
    const double c = b - s1 * (b - a) / (s1 - s0);
    a = b;
    s0 = s1;
    b = c;
    rc = sigma(b, &s1, &w1);
    if (rc != FV_OK) break;
    if (std::fabs(b - a) <= o.rtol * std::fabs(b)) { out = FV_OK; break; }
  }
  if (stats) *stats = st;
  if (rc != FV_OK) return rc;
  *re_cr = b;
  *omega_cr = w1;
  if (out != FV_OK) set_error("fv_critical_re: no convergence within max_iter");
  return out;
}

}  // extern "C"
