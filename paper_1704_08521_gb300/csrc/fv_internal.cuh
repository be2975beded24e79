// Internal declarations of the fvns library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "fvns.h"
#include "fv_ff.cuh"

namespace fv {

// ---------------------------------------------------------------- errors --
void set_error(const std::string& msg);
fv_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define FV_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) return ::fv::cuda_fail(e_, #call, __FILE__, __LINE__); \
  } while (0)

#define FV_CHECK_LAUNCH() FV_CUDA(cudaGetLastError())

#define FV_TRY(call)                      \
  do {                                    \
    fv_status s_ = (call);                \
    if (s_ != FV_OK) return s_;           \
  } while (0)

// ------------------------------------------------------------ metrics ----
// Device view of the 1-D grid metrics (Section 3, Eq. 5 and the finite-volume
// reading): per axis d, for n_d cells,
//   idx[d][m] = 1/dx_m          (m = 0..n-1)
//   idc[d][f] = 1/dc_f          (f = 0..n, half cells at the walls)
//   th[d][f]  = (dx_{f-1}/2)/dc_f   linear-interpolation weight from the
//               centres f-1, f to the face f (f = 1..n-1; 0 at walls)
//   dx[d][m], dc[d][f]          (volumes of the inner product)
template <typename T>
struct Met {
  int n[3];
  int64_t ncell;
  const T* idx[3];
  const T* idc[3];
  const T* th[3];
  const T* dx[3];
  const T* dc[3];
};

// Tensor-product eigenbasis of the Neumann operator D G along one axis.
struct AxisBasis {
  int n = 0;
  int null_index = 0;          // index of the zero eigenvalue
  std::vector<double> lam;     // n
  std::vector<double> E;       // n x n row-major: phi[m] = sum_a E[m][a] phihat[a]
  std::vector<double> Einv;    // n x n row-major: rhat[a] = sum_m Einv[a][m] r[m]
};

// float32 metrics plus the float-float 1/dx of the mixed SIMPLE loop
struct MetFF {
  int n[3];
  int64_t ncell;
  const float* idc[3];
  const float2* idx[3];
  const float2* idcf[3];   // float-float 1/dc (gradient of the FV_FF loop)
};

template <typename T>
struct TpfDev {
  int n[3];
  int null_index[3];
  const T* E[3];
  const T* Einv[3];
  const T* lam[3];
  const T* Et[3];      // transposes (E^T, Einv^T), the k-major operands of
  const T* Einvt[3];   // the fused shared-memory transform kernels
};

// Tensor-core operands of the fused float32 pressure solve (every n <= 128):
// the eigenbases split into TF32 hi + lo parts and stored in the canonical
// K-major layout of fv_tc5.cuh, ready for 16-byte copies into shared memory.
//   bx[dir]: slab_nsplit column chunks, each [hi | lo] of 128 x up8(nx),
//            element (a, i) = M[a0 + a][i] for a < slab_n (M = Einv_x for dir 0,
//            E_x for 1), zero rows beyond
//   ay[dir]: [hi | lo] of 128 x up8(ny), element (b, j) = M[b][j] (Einv_y / E_y)
//   az[0], az[1]: [hi | lo] of 128 x up8(nz) of Einv_z and E_z
struct TcMats {
  bool ready = false;
  int slab_nsplit = 1, slab_n = 0;   // column chunks of the slab kernel, chunk width
  int col_n = 0;                     // (x, y) columns per block of the column kernel
  const float* bx[2] = {nullptr, nullptr};
  const float* ay[2] = {nullptr, nullptr};
  const float* az[2] = {nullptr, nullptr};
};

// device-side state of one SIMPLE loop (graph path)
struct LoopState {
  float phi1, phi_prev, phi_last, div_last;
  int pass, nan, status;        // status: 0 running, 1 converged, 2 pass cap, 3 NaN,
                                // 4 a bounded wait of a pressure transform gave up
  int worst;                    // largest status of the evaluations since graph_take_status
                                // (kept across evaluations: lets drivers launch them
                                // asynchronously and check once per cycle)
};

// one captured, instantiated evaluation graph (per grid and shift sigma)
struct GraphCache {
  bool ready = false;
  double sigma = 0.0;
  int prec = FV_MIXED;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t init_node = nullptr;
  void* d_call = nullptr;
  LoopState* d_loop = nullptr;
};

}  // namespace fv

struct fv_grid {
  int n[3];
  int64_t ncell, nvel;
  int map;
  double alpha, re;
  cudaStream_t stream;

  // host copies
  std::vector<double> h_x[3], h_dx[3], h_dc[3];
  fv::AxisBasis basis[3];

  // device allocations
  void* d_met_d = nullptr;   // double metrics (packed)
  void* d_met_f = nullptr;   // float metrics
  void* d_tpf_d = nullptr;   // double E/Einv/lam
  void* d_tpf_f = nullptr;   // float E/Einv/lam
  fv::Met<double> met_d;
  fv::Met<float> met_f;
  fv::TpfDev<double> tpf_d;
  fv::TpfDev<float> tpf_f;
  void* d_tc = nullptr;      // tensor-core operands of the fused pressure solve
  fv::TcMats tc;

  // workspace
  double* vel_buf[3] = {nullptr, nullptr, nullptr};   // n_vel each
  double* cell_buf[3] = {nullptr, nullptr, nullptr};  // n_cell each
  void* tpf_buf[2] = {nullptr, nullptr};              // n_cell doubles each (float use half)
  double* d_scal = nullptr;      // 64 device scalars
  unsigned* d_fault = nullptr;   // sticky: nonzero once a bounded device wait gave up
  double* d_part = nullptr;      // reduction partials
  double* wts = nullptr;         // W: momentum control-volume size per velocity entry
  float2* wts_ff = nullptr;      // W split into float-float pairs
  int64_t part_len = 0;
  double* h_scal = nullptr;      // pinned host mirror of d_scal
  int64_t ws_bytes = 0;

  // mixed-precision workspace (float32 operands, float-float SIMPLE state)
  float* U32 = nullptr;          // n_vel
  float* x32 = nullptr;          // n_vel
  float* w32 = nullptr;          // n_vel
  float2* vff[2] = {nullptr, nullptr};   // n_vel each
  float2* pff = nullptr;         // n_cell
  float* r32 = nullptr;          // n_cell
  float* phi32 = nullptr;        // n_cell
  void* d_met_ff = nullptr;      // float-float 1/dx per axis
  fv::MetFF met_ff;
  // float-float metrics and operands of the FV_FF J.v
  void* d_met_fn = nullptr;
  fv::Met<fv::ffn> met_fn;
  float2* Uff = nullptr;         // n_vel
  float2* xff = nullptr;         // n_vel
  // registered base flow (fv_grid_set_base): U32 / Uff hold its rounding and
  // split, base_ptr the caller's float64 array (used by the FP64 form)
  const double* base_ptr = nullptr;

  // captured evaluation graphs of the mixed path (built on first use)
  fv::GraphCache graphs[4];
  mutable bool capturing = false;
  bool use_graph = true;          // FVNS_NO_GRAPH=1 selects the host-driven loop

  // optional per-kernel-class event timing
  mutable bool prof_on = false;
  mutable std::vector<cudaEvent_t> ev_pool;
  mutable std::vector<int> ev_kind;     // kind of each recorded (start, stop) pair
  mutable size_t ev_used = 0;

  // Stokes preconditioner of the Newton corrections (built on first use)
  void* d_helm = nullptr;        // per axis: face and cell eigenbases, scaled eigenvalues
  fv::TpfDev<float> helm[3];     // per velocity component
  std::vector<double> helm_lam[3][2];   // raw 1-D eigenvalues per axis (0 face, 1 cell)
  double helm_sigma = -1.0, helm_re = -1.0;

  // Krylov basis (allocated on first use)
  double* kry = nullptr;
  int kry_cols = 0;
  double* kry_small = nullptr;   // device small-matrix area
  void* d_arn = nullptr;         // device Arnoldi area: the cycle's Hessenberg H, a scale

  // multigrid pressure solve: hierarchy, level arrays, CG vectors (first use)
  void* mg = nullptr;
};

namespace fv {

// scalar slots in d_scal
enum {
  S_PHI_MAX = 0,   // max |phi| of the last SIMPLE pass (as uint64 bits)
  S_DIV_MAX = 1,   // max |D v|
  S_NAN = 2,       // nonzero when a NaN was seen
  S_PHI_MAX_F = 3, // float max |phi| (bits in the low word) of the mixed loop
  S_DIV_MAX_F = 4, // float max |D v| of the mixed loop
  S_RED = 8        // start of general reduction results (56 slots)
};
constexpr int kScalars = 64;

// ------------------------------------------------------- instrumentation -
// Every launch goes through LaunchScope: it counts the launch and, when the
// grid's profiler is on, brackets it with CUDA events on the grid's stream.
void count_launch();
struct LaunchScope {
  const fv_grid* g;
  int kind;
  size_t idx;
  LaunchScope(const fv_grid* g_, int kind_);
  ~LaunchScope();
};

// Cell-kernel launch shape: 256 threads tile the x-y plane linearly (x
// fastest, so a warp reads consecutive addresses) and every thread marches
// over kCellKz consecutive z-planes; ~nx*ny*nz/1024 blocks of real work.
constexpr int kCellThreads = 256;
constexpr int kCellKz = 4;
inline dim3 cell_launch_grid(const int n[3]) {
  const int64_t plane = (int64_t)n[0] * n[1];
  return dim3((unsigned)((plane + kCellThreads - 1) / kCellThreads),
              (unsigned)((n[2] + kCellKz - 1) / kCellKz), 1);
}

// ------------------------------------------------------------- kernels ---
// all launches are on g->stream; they return FV_OK or FV_ECUDA
fv_status launch_momentum_jac(const fv_grid* g, const double* U, const double* v, double* out,
                              int prec, double shift);
fv_status launch_residual(const fv_grid* g, const double* U, const double* P,
                          double* Fm, double* Fdiv);
fv_status launch_divergence(const fv_grid* g, const double* v, double* r, double* maxabs_slot);
// vout = vin - omega G phi (faces), p += omega phi (p may be null),
// r = D vout, max|phi| and max|r| into the scalar slots (reset by caller)
fv_status launch_correct_div(const fv_grid* g, const double* vin, double* vout,
                             const void* phi, bool phi_is_float, double* p, double* r,
                             double omega);
fv_status launch_zero_walls(const fv_grid* g, double* v);

// mixed-precision path (fv_mixed.cu)
// J.v tiled kernels (fv_jv.cuh): U from Ud (float64) or, when null, the
// grid's registered base flow (U32 / Uff); x float64; call (graph launches):
// a device block whose first two members are the U and x pointers
fv_status launch_jv_f32(const fv_grid* g, const double* Ud, const double* x, float* out,
                        double shift, const void* call = nullptr);
fv_status launch_jv_f32_out64(const fv_grid* g, const double* Ud, const double* x, double* out,
                              double shift);
fv_status launch_jv_ff(const fv_grid* g, const double* Ud, const double* x, float2* out,
                       double shift, const void* call = nullptr);
fv_status launch_jv_ff_out64(const fv_grid* g, const double* Ud, const double* x, double* out,
                             double shift);
fv_status launch_round_f32(const fv_grid* g, const double* in, float* out, int64_t n);
fv_status launch_div_f32(const fv_grid* g, const float* w32, float* r32);
// one float-float SIMPLE pass; first: vin is the float32 w, p starts at 0
fv_status launch_correct_ff(const fv_grid* g, bool first, const void* vin, float2* vout,
                            const float* phi, float2* p, float* r, double omega, bool ffg = false);
// out = hi + lo (- sigma * x) as float64; p_out = p_ff
fv_status launch_join_ff(const fv_grid* g, const float2* v, const double* x, double sigma,
                         double* out, int64_t n);
fv_status launch_join_ff_cells(const fv_grid* g, const float2* p, double* out);
fv_status launch_widen_f32(const fv_grid* g, const float* in, double* out, int64_t n);

// FV_FF operands and stencil (fv_mixed.cu)
fv_status launch_split_ff(const fv_grid* g, const double* in, float2* out, int64_t n);
// register U as the grid's base flow: U32 = round(U), Uff = split(U)
fv_status set_base(fv_grid* g, const double* U);
fv_status launch_div_ff(const fv_grid* g, const float2* w, float* r32);

// graph path (fv_graph.cu): one mixed-precision Krylov-vector evaluation as
// one graph launch; with sync, the loop statistics are read back.
fv_status mixed_krylov_graph(const fv_grid* g, const double* U, const double* x, double* out,
                             double* p, double sigma, double eps, int max_pass, double omega,
                             bool sync, int* passes, double* phi1, double* phil, double* divl,
                             int* status, int prec = FV_MIXED);
void destroy_graph_cache(GraphCache& c);

// tensor-product pressure solve: phi = (D G)^+ r ; phi is float or double
fv_status tpf_solve(const fv_grid* g, const double* r, void* phi, int prec);
fv_status tpf_solve_f32(const fv_grid* g, const float* r, float* phi);
// one float64 1-D transform along `axis` with the matrix M (n x n, row-major)
fv_status transform_axis_f64(const fv_grid* g, int axis, const double* M, const double* in,
                             double* out);
// the unfused float32 transforms with the tables and eigenvalues of tp
// (scaling by 1 / (lam_z + lam_y + lam_x); null_index -1: no null mode)
fv_status tpf_run_f32(const fv_grid* g, const TpfDev<float>& tp, const float* r, float* phi);
// right preconditioner of the Newton corrections (fv_precond.cu):
// out = P (sigma_p - Lap / Re)^-1 y, float32 transforms, float-float projection
fv_status stokes_precond_apply(fv_grid* g, const double* y, double* out, double sigma_p);
// out = P (g->w32): the mixed SIMPLE loop from the float32 field in g->w32
// (divergence in g->r32) to a relative correction eps (fv_krylov.cu)
fv_status simple_project_w32(const fv_grid* g, double* out, double eps);
void destroy_stokes_tables(fv_grid* g);
// builds g->tc when every dimension is <= 128 (fv_poisson.cu)
fv_status build_tc_mats(fv_grid* g);

// learned first pass of the SIMPLE loop (fv_unet.cu): phi = guess for r
fv_status unet_guess_f32(fv_unet* u, const fv_grid* g, const float* r, float* phi);
// max |x[0..n)| of a float32 array to the host (synchronises g's stream)
fv_status absmax_f32_host(const fv_grid* g, const float* x, int64_t n, double* out);
fv_status tpf_one_transform_f32(const fv_grid* g, int axis);

// the largest status (1 converged, 2 pass cap, 3 NaN, 4 timeout; 0 none) of
// the graph evaluations on g since the last call, then reset (synchronises
// g's stream); with_fault = false leaves the sticky timeout word alone (it
// stays pending until an evaluation reports it)
fv_status graph_take_status(fv_grid* g, int* worst, bool with_fault = true);
// read and clear g's sticky timeout word (synchronises g's stream)
fv_status take_fault(const fv_grid* g, bool* hit);
// the fv_status of an evaluation status (0/1 -> FV_OK) with its message
fv_status status_error(int status);
// fill g->wts and g->wts_ff (the W of the inner products; 0 on wall faces)
fv_status fill_face_weights(fv_grid* g);
// vector kernels (weighted inner products, Gram-Schmidt); ff_arith: the
// float-float form on the FP32 pipes (about 2^-46 relative per term) used for
// the Krylov bases of the mixed and float-float precisions, else FP64
fv_status vec_dots(const fv_grid* g, const double* V, int64_t ldv, int nvec, const double* w,
                   double* d_out /* nvec, device */, bool ff_arith = false);
fv_status vec_update(const fv_grid* g, double* w, const double* V, int64_t ldv, int nvec,
                     const double* d_h, double sign, bool ff_arith = false);
fv_status vec_axpby(const fv_grid* g, int64_t n, double a, const double* x, double b,
                    const double* y, double* out);
fv_status vec_scale_by_device(const fv_grid* g, int64_t n, const double* x, const double* d_s,
                              int mode, double* out);
fv_status vec_combine(const fv_grid* g, const double* V, int64_t ldv, int nin,
                      const double* d_C /* nin x nout, row-major */, int nout, double* out,
                      int64_t ldo, bool ff_arith = false);
fv_status vec_maxabs(const fv_grid* g, int64_t n, const double* x, double* slot);
fv_status widen_float(const fv_grid* g, const float* src, double* dst, int64_t n);

// scalar helpers
fv_status reset_scalars(const fv_grid* g);
fv_status fetch_scalars(const fv_grid* g, double* host /* kScalars */);
double bits_to_double(double slot);

// small dense linear algebra (host), used by the GMRES / Arnoldi drivers
// H is m x m row-major upper Hessenberg.
bool hess_eigenvalues(int m, const double* H, double* wr, double* wi);
bool host_axis_tables(int n, int map, AxisBasis& B);
// eigen-decomposition of the symmetric tridiagonal (d, e): lam, Z (n x n
// row-major, eigenvectors as columns); implicit QR with Wilkinson shifts
// faces x_0..x_n of an axis with n cells under the stretching map
std::vector<double> map_faces(int n, int map);

// multigrid pressure solve (built on first use, freed with the grid)
fv_status mg_solve(fv_grid* g, const double* r, double* phi, const double* guess,
                   const fv_mg_opts& o, fv_mg_stats* stats);
void destroy_mg(fv_grid* g);

bool sym_tridiag_eig(int n, const std::vector<double>& d, const std::vector<double>& e,
                     std::vector<double>& lam, std::vector<double>& Z);

// one implicit double-shift step with the shift pair re +- i im (Q accumulated)
void francis_double_step(int m, double* H, double* Q, double re, double im);
void single_shift_step(int m, double* H, double* Q, double mu);
// y (complex, m) with (H - theta I) y ~ 0, unit 2-norm
void hess_eigvec(int m, const double* H, double tr, double ti, double* yr, double* yi);
}  // namespace fv
