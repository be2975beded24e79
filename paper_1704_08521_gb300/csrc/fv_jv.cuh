// Tiled, z-marching J.v (Eq. 10 / the linearised momentum operator of Eq. 6)
// in flux form, shared by the float32, float-float and float64 forms.
//
// Each momentum control volume's balance is a difference of fluxes through
// its faces; every such flux is shared by two neighbouring control volumes.
// The kernel therefore computes, per cell (fi, fj, k) and per plane, the nine
// fluxes G through the LOW faces of the three control volumes owned by the
// cell (u on x-face fi, v on y-face fj, w on z-face k), each G = (1/Re) D - C
// (diffusive minus convective flux), and forms every balance as
//   w_c = sum_d (G_cd(high) - G_cd(low)) / (width of the CV along d) + shift q_c,
// where the high flux of one cell is the low flux of its neighbour:
//   x-neighbour and y-neighbour fluxes are exchanged through shared memory,
//   the z-flux of the face above is computed one plane ahead and carried in
//   registers while the block marches up its chunk of planes.
//
// Fluxes (JAC form, homogeneous walls; U base, Q perturbation, at the face of
// the control volume in the named direction):
//   centre fluxes (normal direction, between faces f-1 and f):
//     D = (Q_f - Q_{f-1}) / dx_{f-1},   C = (U_{f-1} + U_f)(Q_{f-1} + Q_f) / 2
//   edge fluxes (tangential direction d of component c):
//     D = (Q_c(e) - Q_c(e-1)) / dc_d(e)        (half cell at a wall)
//     C = the linearised product of the two interpolated velocities at the
//         edge, the same for both components that share it:
//         E_xy = I_y(U_u) I_x(Q_v) + I_y(Q_u) I_x(U_v)   (u along y = v along x)
//         E_xz = I_z(U_u) I_x(Q_w) + I_z(Q_u) I_x(U_w)
//         E_yz = I_z(U_v) I_y(Q_w) + I_z(Q_v) I_y(U_w)
//     with I_d(F) = F(e-1) + th_d(e) (F(e) - F(e-1)), the distance-weighted
//     interpolation to the edge; wall-normal velocities are zero, so every
//     convective wall flux vanishes and corner values never enter.
// Values outside the domain (beyond a wall) load as zero: the homogeneous
// wall value of the diffusive flux, and a zero transport velocity.
//
// Block: one thread per cell of the (TXo + 2) x (TYo + 2) tile (the outputs
// and a one-cell halo); each thread copies and converts its own cell of every
// plane.  The threads of the (TXo + 1) x (TYo + 1) cells past the low halo
// row and column compute the fluxes through their cells' low faces, and the
// TXo x TYo of them whose high neighbours are in the tile form the outputs.
// Shared memory: two plane slots of the six fields on the tile and the
// exchanged x/y fluxes.  Raw planes arrive through a cp.async ring issued
// three planes ahead.
// U is read in its stored form (the grid's registered base flow, walls
// zeroed); x is the caller's float64 vector, rounded / split when a plane is
// converted.
#pragma once

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {
namespace jv {

struct Tile {
  int txo, tyo, kz;      // outputs per block in x, y; planes per block
};

// value types: arithmetic T, stored base flow TU, output TO
template <typename T> __device__ __forceinline__ T from_f64(double d);
template <> __device__ __forceinline__ float from_f64<float>(double d) { return f64_round_f32(d); }
template <> __device__ __forceinline__ double from_f64<double>(double d) { return d; }
template <> __device__ __forceinline__ ffn from_f64<ffn>(double d) { return ffn(f64_split(d)); }

template <typename T, typename TU> __device__ __forceinline__ T from_store(TU v);
template <> __device__ __forceinline__ float from_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double from_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ ffn from_store<ffn, float2>(float2 v) { return ffn(v); }

template <typename T, typename TO> __device__ __forceinline__ TO to_store(T v);
template <> __device__ __forceinline__ float to_store<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double to_store<float, double>(float v) { return f32_to_f64(v); }
template <> __device__ __forceinline__ double to_store<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float2 to_store<ffn, float2>(ffn v) { return make_float2(v.hi, v.lo); }
template <> __device__ __forceinline__ double to_store<ffn, double>(ffn v) { return ff_join(v.hi, v.lo); }

// Pointers of one launch: Ur the base flow in its stored form (float32
// rounding, float-float split or float64), x the float64 perturbation; when
// `call` is given (graph launches) x is read from it.
struct CallPtrs {
  const double* U;
  const double* x;
};

template <typename T, typename TU, typename TO>
struct Args {
  Met<T> m;
  const TU* Ur;
  const double* x;
  TO* out;
  const CallPtrs* call;
  T inv_re, shift;
  Tile t;
};

// six fields in a plane slot: U_u, U_v, U_w, Q_u, Q_v, Q_w
enum { UU = 0, UV = 1, UW = 2, QU = 3, QV = 4, QW = 5 };

// raw -> arithmetic conversion of one plane cell value
template <typename T, typename R> __device__ __forceinline__ T conv(R v);
template <> __device__ __forceinline__ float conv<float, double>(double v) { return f64_round_f32(v); }
template <> __device__ __forceinline__ float conv<float, float>(float v) { return v; }
template <> __device__ __forceinline__ double conv<double, double>(double v) { return v; }
template <> __device__ __forceinline__ ffn conv<ffn, double>(double v) { return ffn(f64_split(v)); }
template <> __device__ __forceinline__ ffn conv<ffn, float2>(float2 v) { return ffn(v); }

// asynchronous global -> shared copy of an 8- or 4-byte value; zero fill
// when !valid (the source is not read)
template <int B>
__device__ __forceinline__ void cp_async_v(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "n"(B), "r"(valid ? B : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Raw planes travel through a ring of kRing shared-memory stages (U in its
// stored type, x as float64), issued kRing planes ahead of their use with
// cp.async (no registers held), and are converted -- float64 rounding or
// splitting, wall entries zeroed -- into two arithmetic slots: the plane being
// computed and the plane above it.
constexpr int kRing = 3;

constexpr int kJvMaxThreads = 320;   // threads (= tile cells) per block, at most

// resident blocks per SM the register budget is sized for: three for the
// float32 form (63 registers), two for the float64 and float-float forms,
// whose fluxes need more registers
template <typename T> struct MinBlocks { static constexpr int value = 3; };
template <> struct MinBlocks<double> { static constexpr int value = 2; };
template <> struct MinBlocks<ffn> { static constexpr int value = 2; };

template <typename T, typename TU, typename TO>
__global__ void __launch_bounds__(kJvMaxThreads, MinBlocks<T>::value) k_jv_tile(Args<T, TU, TO> a) {
  extern __shared__ __align__(16) unsigned char jv_smem[];
  const Met<T>& m = a.m;
  const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
  const int nc = (int)m.ncell;
  const int TXo = a.t.txo, TYo = a.t.tyo;
  const int LX = TXo + 2, LY = TYo + 2, LXY = LX * LY;
  const int nthr = blockDim.x;                               // == LXY
  const int tid = threadIdx.x;
  const int li = tid % LX, lj = tid / LX;                    // this thread's tile cell
  const int tx = li - 1, ty = lj - 1;                        // its flux position
  const bool flux_thr = li >= 1 && lj >= 1;
  const int i0 = blockIdx.x * TXo, j0 = blockIdx.y * TYo;
  const int k0 = blockIdx.z * a.t.kz;
  const int k1 = min(k0 + a.t.kz, nz);
  const int fi = i0 + tx, fj = j0 + ty;                     // flux position
  // shared layout: raw ring [kRing][3 U (TU) | 3 x (double)] x LXY, two
  // arithmetic slots [6][LXY] of T, exchanged fluxes [2][3][nthr] of T
  const size_t xbytes = 3 * (size_t)LXY * sizeof(double);
  const size_t stage = xbytes + ((3 * (size_t)LXY * sizeof(TU) + 15) & ~(size_t)15);
  auto rx = [&](int st) { return reinterpret_cast<double*>(jv_smem + st * stage); };
  auto ru = [&](int st) { return reinterpret_cast<TU*>(jv_smem + st * stage + xbytes); };
  T* slot0 = reinterpret_cast<T*>(jv_smem + kRing * stage);
  T* slot1 = slot0 + 6 * LXY;
  T* gxs = slot1 + 6 * LXY;                                  // [3][nthr]
  T* gys = gxs + 3 * nthr;                                   // [3][nthr]

  const double* X = a.x;
  if (a.call) X = a.call->x;
  const TU* Ur = a.Ur;

  // this thread's tile cell in the plane
  const int ci = i0 - 1 + li, cj = j0 - 1 + lj;
  const bool cin = ci >= 0 && ci < nx && cj >= 0 && cj < ny;
  const int cb = cin ? cj * nx + ci : 0;
  auto issue = [&](int k) {                 // plane k -> ring stage (k + 1) % kRing
    const int st = (k + 1 + kRing) % kRing;
    const bool v = cin && k >= 0 && k < nz;
    const int b = v ? k * (nx * ny) + cb : 0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cp_async_v<sizeof(TU)>(ru(st) + c * LXY + tid, Ur + c * nc + b, v);
      cp_async_v<8>(rx(st) + c * LXY + tid, X + c * nc + b, v);
    }
    cp_async_commit();
  };
  auto convert = [&](int k, T* s) {         // ring stage of plane k -> slot s (walls zero)
    const int st = (k + 1 + kRing) % kRing;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const bool wall = (c == 0 && ci == 0) || (c == 1 && cj == 0) || (c == 2 && k == 0);
      s[c * LXY + tid] = wall ? T(0) : conv<T, TU>(ru(st)[c * LXY + tid]);
      s[(3 + c) * LXY + tid] = wall ? T(0) : conv<T, double>(rx(st)[c * LXY + tid]);
    }
  };
  // wait until plane k's copies (issued before the `newer` later planes) landed
  auto wait_for = [&](int newer) {
    if (newer >= 2) cp_async_wait<2>();
    else if (newer == 1) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
  };

  // tile offsets of this thread's position and its low neighbours
  const int o0 = tid;
  // low neighbours; the halo row / column threads read their own cell instead
  // (their fluxes are computed but never read)
  const int oxm = flux_thr ? o0 - 1 : o0, oym = flux_thr ? o0 - LX : o0;

  // per-thread metrics (x from fi, y from fj; clamped where unused)
  const int fic = min(max(fi, 0), nx), fjc = min(max(fj, 0), ny);
  const T idc_x = m.idc[0][fic], th_x = m.th[0][fic];
  const T idxm_x = m.idx[0][max(fic - 1, 0)];
  const T idx_x = m.idx[0][min(fic, nx - 1)];
  const T idc_y = m.idc[1][fjc], th_y = m.th[1][fjc];
  const T idxm_y = m.idx[1][max(fjc - 1, 0)];
  const T idx_y = m.idx[1][min(fjc, ny - 1)];
  const T inv_re = a.inv_re;
  const T half = T(0.5);

  const bool out_thr = flux_thr && tx < TXo && ty < TYo && fi < nx && fj < ny;

  // z-fluxes through the face between planes kf - 1 (below, "zm") and kf
  // ("cz" = own column values of plane kf); the w neighbours along x and y
  // come from the slot of plane kf
  auto zflux = [&](const T (&cz)[6], const T (&zm)[6], const T* sup, int kf, T (&gz)[3],
                   T (&ez)[2]) {
    const int kfc = min(kf, nz);
    const T idc_z = m.idc[2][kfc], th_z = m.th[2][kfc];
    const T idxm_z = m.idx[2][max(kfc - 1, 0)];
    const T Uwxm = sup[UW * LXY + oxm], Qwxm = sup[QW * LXY + oxm];
    const T Uwym = sup[UW * LXY + oym], Qwym = sup[QW * LXY + oym];
    const T Iz_Uu = zm[UU] + th_z * (cz[UU] - zm[UU]);
    const T Iz_Qu = zm[QU] + th_z * (cz[QU] - zm[QU]);
    const T Iz_Uv = zm[UV] + th_z * (cz[UV] - zm[UV]);
    const T Iz_Qv = zm[QV] + th_z * (cz[QV] - zm[QV]);
    const T Ix_Uw = Uwxm + th_x * (cz[UW] - Uwxm);
    const T Ix_Qw = Qwxm + th_x * (cz[QW] - Qwxm);
    const T Iy_Uw = Uwym + th_y * (cz[UW] - Uwym);
    const T Iy_Qw = Qwym + th_y * (cz[QW] - Qwym);
    const T Exz = Iz_Uu * Ix_Qw + Iz_Qu * Ix_Uw;
    const T Eyz = Iz_Uv * Iy_Qw + Iz_Qv * Iy_Uw;
    ez[0] = Exz;
    ez[1] = Eyz;
    gz[0] = inv_re * ((cz[QU] - zm[QU]) * idc_z) - Exz;
    gz[1] = inv_re * ((cz[QV] - zm[QV]) * idc_z) - Eyz;
    gz[2] = inv_re * ((cz[QW] - zm[QW]) * idxm_z) - half * (zm[UW] + cz[UW]) * (zm[QW] + cz[QW]);
  };

  // ---- chunk start: planes k0 - 1 and k0, the z-flux of face k0, then k0 + 1
  T own[6], gz_lo[3], gz_hi[3], ez_lo[2], ez_hi[2];
  issue(k0 - 1);
  issue(k0);
  issue(k0 + 1);
  wait_for(2);
  convert(k0 - 1, slot0);
  wait_for(1);
  convert(k0, slot1);
  __syncthreads();
  issue(k0 + 2);                            // ring stage of k0 - 1 is free
  {
    T below[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      below[f] = slot0[f * LXY + o0];
      own[f] = slot1[f * LXY + o0];
    }
    zflux(own, below, slot1, k0, gz_lo, ez_lo);
  }
  __syncthreads();                          // slot0 (plane k0 - 1) is free
  wait_for(1);                              // plane k0 + 1 (k0 + 2 still in flight)
  convert(k0 + 1, slot0);
  __syncthreads();
  issue(k0 + 3);
  int last = k0 + 3;                        // last plane issued
  T* sc = slot1;                            // plane k
  T* sn = slot0;                            // plane k + 1

  for (int k = k0; k < k1; ++k) {
    // x / y fluxes of plane k through the low faces of this position
    const T Uuxm = sc[UU * LXY + oxm], Quxm = sc[QU * LXY + oxm];
    const T Uvxm = sc[UV * LXY + oxm], Qvxm = sc[QV * LXY + oxm];
    const T Qwxm = sc[QW * LXY + oxm];
    const T Uuym = sc[UU * LXY + oym], Quym = sc[QU * LXY + oym];
    const T Uvym = sc[UV * LXY + oym], Qvym = sc[QV * LXY + oym];
    const T Qwym = sc[QW * LXY + oym];
    const T Iy_Uu = Uuym + th_y * (own[UU] - Uuym);
    const T Iy_Qu = Quym + th_y * (own[QU] - Quym);
    const T Ix_Uv = Uvxm + th_x * (own[UV] - Uvxm);
    const T Ix_Qv = Qvxm + th_x * (own[QV] - Qvxm);
    const T Exy = Iy_Uu * Ix_Qv + Iy_Qu * Ix_Uv;
    T gx[3], gy[3];
    gx[0] = inv_re * ((own[QU] - Quxm) * idxm_x) - half * (Uuxm + own[UU]) * (Quxm + own[QU]);
    gx[1] = inv_re * ((own[QV] - Qvxm) * idc_x) - Exy;
    gy[0] = inv_re * ((own[QU] - Quym) * idc_y) - Exy;
    gy[1] = inv_re * ((own[QV] - Qvym) * idxm_y) - half * (Uvym + own[UV]) * (Qvym + own[QV]);
    // w through the x- and y-faces of its control volume: the edges of face
    // k, whose convective products came with the z-fluxes of that face
    gx[2] = inv_re * ((own[QW] - Qwxm) * idc_x) - ez_lo[0];
    gy[2] = inv_re * ((own[QW] - Qwym) * idc_y) - ez_lo[1];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      gxs[c * nthr + tid] = gx[c];
      gys[c * nthr + tid] = gy[c];
    }
    // z-fluxes through the face k + 1 (top of this plane)
    T above[6];
#pragma unroll
    for (int f = 0; f < 6; ++f) above[f] = sn[f * LXY + o0];
    zflux(above, own, sn, k + 1, gz_hi, ez_hi);
    __syncthreads();
    if (out_thr) {
      const int hx = tid + 1, hy = tid + LX;        // high x / y neighbours in the tile
      const T idx_z = m.idx[2][k], idc_z = m.idc[2][k];
      const int b = (k * ny + fj) * nx + fi;
      T wu = T(0), wv = T(0), ww = T(0);
      if (fi > 0)
        wu = (gxs[0 * nthr + hx] - gx[0]) * idc_x + (gys[0 * nthr + hy] - gy[0]) * idx_y +
             (gz_hi[0] - gz_lo[0]) * idx_z + a.shift * own[QU];
      if (fj > 0)
        wv = (gxs[1 * nthr + hx] - gx[1]) * idx_x + (gys[1 * nthr + hy] - gy[1]) * idc_y +
             (gz_hi[1] - gz_lo[1]) * idx_z + a.shift * own[QV];
      if (k > 0)
        ww = (gxs[2 * nthr + hx] - gx[2]) * idx_x + (gys[2 * nthr + hy] - gy[2]) * idx_y +
             (gz_hi[2] - gz_lo[2]) * idc_z + a.shift * own[QW];
      a.out[b] = to_store<T, TO>(wu);
      a.out[nc + b] = to_store<T, TO>(wv);
      a.out[2 * nc + b] = to_store<T, TO>(ww);
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) gz_lo[c] = gz_hi[c];
    ez_lo[0] = ez_hi[0];
    ez_lo[1] = ez_hi[1];
#pragma unroll
    for (int f = 0; f < 6; ++f) own[f] = above[f];
    if (k + 1 < k1) {
      // plane k + 2 replaces plane k in its slot; the plane kRing ahead of it
      // goes into the ring stage it leaves.  No barrier before the
      // conversion: every thread converts exactly the ring cells whose
      // copies it issued (its own cp.async wait covers them), nobody reads
      // slot sc after the flux barrier above, and the barrier below orders
      // this plane's output reads of gxs / gys before the next plane's writes
      const int newer = last - (k + 2);
      if (newer >= 2) cp_async_wait<2>();
      else if (newer == 1) cp_async_wait<1>();
      else cp_async_wait<0>();
      convert(k + 2, sc);
      if (last + 1 <= k1) {
        issue(last + 1);
        ++last;
      } else {
        cp_async_commit();                           // empty group keeps the counting uniform
        ++last;
      }
      __syncthreads();
      T* t = sc;
      sc = sn;
      sn = t;
    }
  }
  cp_async_wait<0>();
}

// Launch shape of a grid: tiles of at most kJvMaxThreads cells (outputs plus
// the one-cell halo) sized to split nx and ny evenly (little idle tail), and
// z-chunks so that the blocks fill the resident slots of the 152 SMs
// (`per_sm` blocks each) once: a second partial wave would double the time
// of the chunk.

inline Tile tile_shape(const int n[3], int per_sm = 3) {
  Tile t;
  const int ntx = (n[0] + 30) / 31;                  // at most 31 outputs (33 cells) along x
  t.txo = (n[0] + ntx - 1) / ntx;
  const int ly_max = kJvMaxThreads / (t.txo + 2);    // tile rows, halo included
  const int nty = (n[1] + ly_max - 3) / (ly_max - 2);
  t.tyo = (n[1] + nty - 1) / nty;
  const int64_t xy = (int64_t)ntx * nty;
  const int64_t slots = 152 * (int64_t)(per_sm < 1 ? 1 : per_sm);
  int chunks = (int)(slots / xy);                    // full waves only
  if (chunks < 1) chunks = 1;
  if (chunks > n[2]) chunks = n[2];
  t.kz = (n[2] + chunks - 1) / chunks;
  return t;
}

inline dim3 tile_grid(const int n[3], const Tile& t) {
  return dim3((unsigned)((n[0] + t.txo - 1) / t.txo), (unsigned)((n[1] + t.tyo - 1) / t.tyo),
              (unsigned)((n[2] + t.kz - 1) / t.kz));
}

inline int tile_threads(const Tile& t) { return (t.txo + 2) * (t.tyo + 2); }

template <typename T, typename TU>
inline size_t tile_smem(const Tile& t) {
  const size_t lxy = (size_t)(t.txo + 2) * (t.tyo + 2);
  const size_t ring = kRing * (3 * lxy * sizeof(double) + ((3 * lxy * sizeof(TU) + 15) & ~(size_t)15));
  return ring + sizeof(T) * (2 * 6 * lxy + 6 * (size_t)tile_threads(t));
}

// Launch with the z-chunks sized by the kernel's measured residency.
template <typename T, typename TU, typename TO>
inline cudaError_t launch(Args<T, TU, TO> a, cudaStream_t s) {
  static bool attr = false;   // per instantiation
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_jv_tile<T, TU, TO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  Tile t = tile_shape(a.m.n);
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jv_tile<T, TU, TO>,
                                                                tile_threads(t), tile_smem<T, TU>(t));
  if (e != cudaSuccess) return e;
  t = tile_shape(a.m.n, per_sm);
  a.t = t;
  k_jv_tile<T, TU, TO><<<tile_grid(a.m.n, t), tile_threads(t), tile_smem<T, TU>(t), s>>>(a);
  return cudaGetLastError();
}

}  // namespace jv
}  // namespace fv
