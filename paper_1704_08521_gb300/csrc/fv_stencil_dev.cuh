// Device stencil of the linearised momentum operator (Eq. 6 / Eq. 10) and of
// the steady momentum residual (Eqs. 1-4), shared by the per-grid kernels
// (fv_stencil.cu) and the batched work-queue kernel (fv_graph.cu).
#pragma once

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {
namespace stencil {

// load an input value in the arithmetic type T; double -> float goes through
// the integer rounding of fv_ff.cuh, not the (slow on GB300) FP64 converter
template <typename T, typename TI>
__device__ __forceinline__ T ld(const TI* __restrict__ p, int i) {
  if constexpr (sizeof(T) == sizeof(TI)) return __ldg(p + i);
  else return T(__ldg(p + i));
}

template <typename T, typename TO>
__device__ __forceinline__ TO to_out(T v) {
  if constexpr (sizeof(T) == 4 && sizeof(TO) == 8) return f32_to_f64(v);
  else return TO(v);
}

// Momentum balance of component C at the face owned by cell (i, j, k).
// JAC: (1/Re) Lap v - div(U (x) v) - div(v (x) U) + shift v   (homogeneous walls)
// else: (1/Re) Lap U - div(U (x) U)                            (lid wall values)
template <typename T, int C, bool JAC, typename TI>
__device__ __forceinline__ T momentum_face(const Met<T>& m, const TI* __restrict__ U,
                                           const TI* __restrict__ V, int base,
                                           const int (&pos)[3], const int (&st)[3],
                                           T inv_re, T lid_hi, T shift) {
  // 32-bit offsets: the API guarantees 3 nx ny nz < 2^31
  const int nc = (int)m.ncell;
  const TI* Uc = U + C * nc;
  const TI* Qc = (JAC ? V : U) + C * nc;
  const int f = pos[C];
  const int nC = m.n[C];

  // ---- direction d = C (normal to the face): values on faces f-1, f, f+1
  const T q0 = ld<T>(Qc, base);
  const T qm = (f > 1) ? ld<T>(Qc, base - st[C]) : T(0);
  const T qp = (f + 1 < nC) ? ld<T>(Qc, base + st[C]) : T(0);
  T diff = ((qp - q0) * m.idx[C][f] - (q0 - qm) * m.idx[C][f - 1]) * m.idc[C][f];
  T conv;
  {
    const T u0 = ld<T>(Uc, base);
    const T um = (f > 1) ? ld<T>(Uc, base - st[C]) : T(0);
    const T up = (f + 1 < nC) ? ld<T>(Uc, base + st[C]) : T(0);
    T Fhi, Flo;
    if (JAC) {
      Fhi = T(0.5) * (u0 + up) * (q0 + qp);
      Flo = T(0.5) * (um + u0) * (qm + q0);
    } else {
      Fhi = T(0.25) * (u0 + up) * (u0 + up);
      Flo = T(0.25) * (um + u0) * (um + u0);
    }
    conv = (Fhi - Flo) * m.idc[C][f];
  }

  // ---- the two tangential directions
#pragma unroll
  for (int t = 1; t <= 2; ++t) {
    const int d = (C + t) % 3;
    const int e = pos[d];
    const int nd = m.n[d];
    // diffusion along d (cell centres e-1, e, e+1; walls at half cells)
    const T wall_hi = (!JAC && d == 2) ? lid_hi : T(0);
    const T sm = (e > 0) ? ld<T>(Qc, base - st[d]) : T(0);
    const T sp = (e + 1 < nd) ? ld<T>(Qc, base + st[d]) : wall_hi;
    diff += ((sp - q0) * m.idc[d][e + 1] - (q0 - sm) * m.idc[d][e]) * m.idx[d][e];

    // convective fluxes through the d-faces e (low) and e+1 (high) of the
    // C-control volume; the transport velocity a_d is interpolated along C
    // from the centres f-1, f; the transported b_C along d from e-1, e.
    const TI* Ud = U + d * nc;
    const TI* Vd = V + d * nc;
    const T thc = m.th[C][f];
    T Flo = T(0), Fhi = T(0);
    if (e > 0) {
      const int b = base;
      const T aU = ld<T>(Ud, b - st[C]) + thc * (ld<T>(Ud, b) - ld<T>(Ud, b - st[C]));
      const T thd = m.th[d][e];
      const T cm = ld<T>(Uc, base - st[d]);
      const T bU = cm + thd * (ld<T>(Uc, base) - cm);
      if (JAC) {
        const T aV = ld<T>(Vd, b - st[C]) + thc * (ld<T>(Vd, b) - ld<T>(Vd, b - st[C]));
        const T bV = sm + thd * (q0 - sm);
        Flo = aU * bV + aV * bU;
      } else {
        Flo = aU * bU;
      }
    }
    if (e + 1 < nd) {
      const int b = base + st[d];
      const T aU = ld<T>(Ud, b - st[C]) + thc * (ld<T>(Ud, b) - ld<T>(Ud, b - st[C]));
      const T thd = m.th[d][e + 1];
      const T c0 = ld<T>(Uc, base);
      const T bU = c0 + thd * (ld<T>(Uc, base + st[d]) - c0);
      if (JAC) {
        const T aV = ld<T>(Vd, b - st[C]) + thc * (ld<T>(Vd, b) - ld<T>(Vd, b - st[C]));
        const T bV = q0 + thd * (sp - q0);
        Fhi = aU * bV + aV * bU;
      } else {
        Fhi = aU * bU;
      }
    }
    conv += (Fhi - Flo) * m.idx[d][e];
  }
  T out = inv_re * diff - conv;
  if (JAC) out += shift * q0;
  return out;
}


}  // namespace stencil
}  // namespace fv
