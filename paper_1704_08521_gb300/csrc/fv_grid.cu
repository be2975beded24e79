// Grid construction: stretched face coordinates (Section 3, Eq. 5), the
// finite-volume metrics, the tensor-product eigenbases of the pressure-
// correction operator (the TPF idea of Section 3) and all workspace.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>

#include "fv_ff.cuh"
#include "fv_internal.cuh"
#include "fvns_host.h"

namespace fv {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

LaunchScope::LaunchScope(const fv_grid* g_, int kind_) : g(g_), kind(kind_), idx(SIZE_MAX) {
  if (g->capturing) return;
  count_launch();
  if (!g->prof_on) return;
  if (g->ev_used + 2 > g->ev_pool.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) { (void)cudaGetLastError(); return; }
      g->ev_pool.push_back(e);
    }
  }
  idx = g->ev_used;
  g->ev_used += 2;
  g->ev_kind.push_back(kind);
  cudaEventRecord(g->ev_pool[idx], g->stream);
}

LaunchScope::~LaunchScope() {
  if (idx != SIZE_MAX) cudaEventRecord(g->ev_pool[idx + 1], g->stream);
}

void set_error(const std::string& msg) { g_last_error = msg; }

fv_status cuda_fail(cudaError_t e, const char* what, const char* file, int line) {
  char buf[512];
  snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  g_last_error = buf;
  return FV_ECUDA;
}

// Face coordinates x_0..x_n of one axis.
std::vector<double> map_faces(int n, int map) {
  std::vector<double> x(n + 1);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i <= n; ++i) {
    double xi = double(i) / double(n);
    if (map == FV_MAP_SINE0975) x[i] = xi - 0.0975 * std::sin(2.0 * pi * xi);   // Eq. 5
    else if (map == FV_MAP_COSINE) x[i] = 0.5 * (1.0 - std::cos(pi * xi));
    else x[i] = xi;
  }
  x[0] = 0.0;
  x[n] = 1.0;
  return x;
}

// Eigen-decomposition of a symmetric tridiagonal matrix (diag d, off-diag e)
// by implicit symmetric QR steps with the Wilkinson shift (Golub & Van Loan,
// Section 8.3).  Z (n x n, row-major) receives the eigenvectors as columns.
static bool tridiag_eig(int n, const std::vector<double>& d, const std::vector<double>& e,
                        std::vector<double>& lam, std::vector<double>& Z) {
  std::vector<double> A((size_t)n * n, 0.0);
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int i = 0; i < n; ++i) a(i, i) = d[i];
  for (int i = 0; i + 1 < n; ++i) a(i, i + 1) = a(i + 1, i) = e[i];
  Z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  const double eps = 2.2204460492503131e-16;
  auto small = [&](int i) {  // is the sub-diagonal entry (i, i-1) negligible?
    return std::fabs(a(i, i - 1)) <= eps * (std::fabs(a(i, i)) + std::fabs(a(i - 1, i - 1)));
  };
  int hi = n - 1;
  int guard = 0;
  while (hi > 0) {
    if (++guard > 60 * n + 100) return false;
    if (small(hi)) { a(hi, hi - 1) = a(hi - 1, hi) = 0.0; --hi; continue; }
    int lo = hi - 1;
    while (lo > 0 && !small(lo)) --lo;
    if (lo > 0) a(lo, lo - 1) = a(lo - 1, lo) = 0.0;
    const double p = a(hi - 1, hi - 1), b = a(hi, hi - 1), q = a(hi, hi);
    const double dd = 0.5 * (p - q);
    const double den = dd + (dd >= 0 ? 1.0 : -1.0) * std::hypot(dd, b);
    const double mu = (den == 0.0) ? q - std::fabs(b) : q - b * b / den;
    double x = a(lo, lo) - mu, z = a(lo + 1, lo);
    for (int k = lo; k < hi; ++k) {
      double r = std::hypot(x, z);
      double cs = 1.0, sn = 0.0;
      if (r != 0.0) { cs = x / r; sn = z / r; }
      const int j0 = (k - 1 > lo) ? k - 1 : lo;
      const int j1 = (k + 2 < hi) ? k + 2 : hi;
      for (int j = j0; j <= j1; ++j) {            // rows k, k+1
        double t0 = a(k, j), t1 = a(k + 1, j);
        a(k, j) = cs * t0 + sn * t1;
        a(k + 1, j) = -sn * t0 + cs * t1;
      }
      for (int i = j0; i <= j1; ++i) {            // columns k, k+1
        double t0 = a(i, k), t1 = a(i, k + 1);
        a(i, k) = cs * t0 + sn * t1;
        a(i, k + 1) = -sn * t0 + cs * t1;
      }
      for (int i = 0; i < n; ++i) {               // Z <- Z R^T
        double t0 = Z[(size_t)i * n + k], t1 = Z[(size_t)i * n + k + 1];
        Z[(size_t)i * n + k] = cs * t0 + sn * t1;
        Z[(size_t)i * n + k + 1] = -sn * t0 + cs * t1;
      }
      if (k + 1 < hi) { x = a(k + 1, k); z = a(k + 2, k); }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = a(i, i);
  return true;
}

bool sym_tridiag_eig(int n, const std::vector<double>& d, const std::vector<double>& e,
                     std::vector<double>& lam, std::vector<double>& Z) {
  return tridiag_eig(n, d, e, lam, Z);
}

// Neumann operator of one axis, L = dx^{-1} T, T symmetric tridiagonal
// (Section 3 step 1, d phi/dn = 0).  Symmetrised S = dx^{-1/2} T dx^{-1/2}.
static bool axis_basis(const std::vector<double>& dx, const std::vector<double>& dc, AxisBasis& B) {
  const int n = (int)dx.size();
  std::vector<double> d(n, 0.0), e(n > 1 ? n - 1 : 1, 0.0);
  for (int f = 1; f < n; ++f) {            // interior face f between cells f-1, f
    const double gco = 1.0 / dc[f];
    d[f - 1] -= gco;
    d[f] -= gco;
    e[f - 1] = gco;
  }
  for (int m = 0; m < n; ++m) d[m] /= dx[m];
  for (int m = 0; m + 1 < n; ++m) e[m] /= std::sqrt(dx[m] * dx[m + 1]);
  std::vector<double> Z;
  if (!tridiag_eig(n, d, e, B.lam, Z)) return false;
  B.n = n;
  B.E.assign((size_t)n * n, 0.0);
  B.Einv.assign((size_t)n * n, 0.0);
  for (int m = 0; m < n; ++m) {
    const double s = std::sqrt(dx[m]);
    for (int a = 0; a < n; ++a) {
      B.E[(size_t)m * n + a] = Z[(size_t)m * n + a] / s;
      B.Einv[(size_t)a * n + m] = Z[(size_t)m * n + a] * s;
    }
  }
  int best = 0;
  for (int a = 1; a < n; ++a)
    if (B.lam[a] > B.lam[best]) best = a;
  B.null_index = best;
  return true;
}

// Tensor-product tables of one axis with n cells and map `map`, on the host
// (used by the allocation-free pressure solve).
bool host_axis_tables(int n, int map, AxisBasis& B) {
  const std::vector<double> x = map_faces(n, map);
  std::vector<double> dx(n), xc(n), dc(n + 1);
  for (int m = 0; m < n; ++m) dx[m] = x[m + 1] - x[m];
  for (int m = 0; m < n; ++m) xc[m] = 0.5 * (x[m] + x[m + 1]);
  dc[0] = 0.5 * dx[0];
  for (int f = 1; f < n; ++f) dc[f] = xc[f] - xc[f - 1];
  dc[n] = 0.5 * dx[n - 1];
  return axis_basis(dx, dc, B);
}

template <typename T>
static fv_status upload_metrics(fv_grid* g, void** dst, Met<T>& met) {
  // layout per axis: idx[n], idc[n+1], th[n+1], dx[n], dc[n+1]
  size_t total = 0;
  for (int d = 0; d < 3; ++d) total += 5 * (size_t)(g->n[d] + 1);
  std::vector<T> h(total, T(0));
  size_t off[3];
  size_t o = 0;
  for (int d = 0; d < 3; ++d) {
    const int n = g->n[d];
    off[d] = o;
    T* p = h.data() + o;
    for (int m = 0; m < n; ++m) p[m] = T(1.0 / g->h_dx[d][m]);
    for (int f = 0; f <= n; ++f) p[(n + 1) + f] = T(1.0 / g->h_dc[d][f]);
    for (int f = 1; f < n; ++f) p[2 * (n + 1) + f] = T(0.5 * g->h_dx[d][f - 1] / g->h_dc[d][f]);
    for (int m = 0; m < n; ++m) p[3 * (n + 1) + m] = T(g->h_dx[d][m]);
    for (int f = 0; f <= n; ++f) p[4 * (n + 1) + f] = T(g->h_dc[d][f]);
    o += 5 * (size_t)(n + 1);
  }
  FV_CUDA(cudaMalloc(dst, total * sizeof(T)));
  g->ws_bytes += total * sizeof(T);
  FV_CUDA(cudaMemcpy(*dst, h.data(), total * sizeof(T), cudaMemcpyHostToDevice));
  T* base = (T*)*dst;
  for (int d = 0; d < 3; ++d) {
    const int n = g->n[d];
    met.n[d] = n;
    met.idx[d] = base + off[d];
    met.idc[d] = base + off[d] + (n + 1);
    met.th[d] = base + off[d] + 2 * (n + 1);
    met.dx[d] = base + off[d] + 3 * (n + 1);
    met.dc[d] = base + off[d] + 4 * (n + 1);
  }
  met.ncell = g->ncell;
  return FV_OK;
}

template <typename T>
static fv_status upload_tpf(fv_grid* g, void** dst, TpfDev<T>& t) {
  size_t total = 0;
  for (int d = 0; d < 3; ++d) total += 4 * (size_t)g->n[d] * g->n[d] + g->n[d];
  std::vector<T> h(total);
  size_t o = 0, offE[3], offI[3], offL[3], offEt[3], offIt[3];
  for (int d = 0; d < 3; ++d) {
    const AxisBasis& B = g->basis[d];
    const int n = B.n;
    const size_t nn = (size_t)n * n;
    offE[d] = o;
    for (size_t q = 0; q < nn; ++q) h[o + q] = T(B.E[q]);
    o += nn;
    offI[d] = o;
    for (size_t q = 0; q < nn; ++q) h[o + q] = T(B.Einv[q]);
    o += nn;
    offEt[d] = o;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) h[o + (size_t)c * n + r] = T(B.E[(size_t)r * n + c]);
    o += nn;
    offIt[d] = o;
    for (int r = 0; r < n; ++r)
      for (int c = 0; c < n; ++c) h[o + (size_t)c * n + r] = T(B.Einv[(size_t)r * n + c]);
    o += nn;
    offL[d] = o;
    for (int a = 0; a < n; ++a) h[o + a] = T(B.lam[a]);
    o += n;
  }
  FV_CUDA(cudaMalloc(dst, total * sizeof(T)));
  g->ws_bytes += total * sizeof(T);
  FV_CUDA(cudaMemcpy(*dst, h.data(), total * sizeof(T), cudaMemcpyHostToDevice));
  T* base = (T*)*dst;
  for (int d = 0; d < 3; ++d) {
    t.n[d] = g->n[d];
    t.null_index[d] = g->basis[d].null_index;
    t.E[d] = base + offE[d];
    t.Einv[d] = base + offI[d];
    t.Et[d] = base + offEt[d];
    t.Einvt[d] = base + offIt[d];
    t.lam[d] = base + offL[d];
  }
  return FV_OK;
}

static fv_status alloc(fv_grid* g, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    set_error(std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
              cudaGetErrorString(e));
    (void)cudaGetLastError();
    return FV_ENOMEM;
  }
  g->ws_bytes += (int64_t)bytes;
  return FV_OK;
}

static fv_status build(fv_grid* g) {
  for (int d = 0; d < 3; ++d) {
    const int n = g->n[d];
    g->h_x[d] = map_faces(n, g->map);
    g->h_dx[d].resize(n);
    for (int m = 0; m < n; ++m) g->h_dx[d][m] = g->h_x[d][m + 1] - g->h_x[d][m];
    std::vector<double> xc(n);
    for (int m = 0; m < n; ++m) xc[m] = 0.5 * (g->h_x[d][m] + g->h_x[d][m + 1]);
    g->h_dc[d].resize(n + 1);
    g->h_dc[d][0] = 0.5 * g->h_dx[d][0];
    for (int f = 1; f < n; ++f) g->h_dc[d][f] = xc[f] - xc[f - 1];
    g->h_dc[d][n] = 0.5 * g->h_dx[d][n - 1];
    if (!axis_basis(g->h_dx[d], g->h_dc[d], g->basis[d])) {
      set_error("tridiagonal eigensolver did not converge");
      return FV_ECUDA;
    }
  }
  FV_TRY(upload_metrics<double>(g, &g->d_met_d, g->met_d));
  FV_TRY(upload_metrics<float>(g, &g->d_met_f, g->met_f));
  FV_TRY(upload_tpf<double>(g, &g->d_tpf_d, g->tpf_d));
  FV_TRY(upload_tpf<float>(g, &g->d_tpf_f, g->tpf_f));
  FV_TRY(build_tc_mats(g));
  for (int i = 0; i < 3; ++i) FV_TRY(alloc(g, (void**)&g->vel_buf[i], g->nvel * sizeof(double)));
  for (int i = 0; i < 3; ++i) FV_TRY(alloc(g, (void**)&g->cell_buf[i], g->ncell * sizeof(double)));
  for (int i = 0; i < 2; ++i) FV_TRY(alloc(g, &g->tpf_buf[i], g->ncell * sizeof(double)));
  // mixed-precision workspace
  FV_TRY(alloc(g, (void**)&g->U32, g->nvel * sizeof(float)));
  FV_TRY(alloc(g, (void**)&g->x32, g->nvel * sizeof(float)));
  FV_TRY(alloc(g, (void**)&g->w32, g->nvel * sizeof(float)));
  for (int i = 0; i < 2; ++i) FV_TRY(alloc(g, (void**)&g->vff[i], g->nvel * sizeof(float2)));
  FV_TRY(alloc(g, (void**)&g->pff, g->ncell * sizeof(float2)));
  FV_TRY(alloc(g, (void**)&g->r32, g->ncell * sizeof(float)));
  FV_TRY(alloc(g, (void**)&g->phi32, g->ncell * sizeof(float)));
  {
    size_t tot = 0;
    for (int d = 0; d < 3; ++d) tot += g->n[d];
    std::vector<float2> h(tot);
    size_t off[3], o = 0;
    for (int d = 0; d < 3; ++d) {
      off[d] = o;
      for (int m = 0; m < g->n[d]; ++m) {
        const ff s = f64_split(1.0 / g->h_dx[d][m]);
        h[o + m] = make_float2(s.hi, s.lo);
      }
      o += g->n[d];
    }
    FV_TRY(alloc(g, &g->d_met_ff, tot * sizeof(float2)));
    FV_CUDA(cudaMemcpy(g->d_met_ff, h.data(), tot * sizeof(float2), cudaMemcpyHostToDevice));
    for (int d = 0; d < 3; ++d) {
      g->met_ff.n[d] = g->n[d];
      g->met_ff.idc[d] = g->met_f.idc[d];
      g->met_ff.idx[d] = (const float2*)g->d_met_ff + off[d];
    }
    g->met_ff.ncell = g->ncell;
  }
  // float-float metrics (FV_FF J.v): idx, idc, th, dx, dc per axis, each
  // value split exactly into (hi, lo)
  {
    size_t total = 0;
    for (int d = 0; d < 3; ++d) total += 5 * (size_t)(g->n[d] + 1);
    std::vector<float2> h(total, make_float2(0.f, 0.f));
    size_t off[3], o = 0;
    auto put = [](double v) { const ff s2 = f64_split(v); return make_float2(s2.hi, s2.lo); };
    for (int d = 0; d < 3; ++d) {
      const int n = g->n[d];
      off[d] = o;
      float2* q = h.data() + o;
      for (int m = 0; m < n; ++m) q[m] = put(1.0 / g->h_dx[d][m]);
      for (int f = 0; f <= n; ++f) q[(n + 1) + f] = put(1.0 / g->h_dc[d][f]);
      for (int f = 1; f < n; ++f) q[2 * (n + 1) + f] = put(0.5 * g->h_dx[d][f - 1] / g->h_dc[d][f]);
      for (int m = 0; m < n; ++m) q[3 * (n + 1) + m] = put(g->h_dx[d][m]);
      for (int f = 0; f <= n; ++f) q[4 * (n + 1) + f] = put(g->h_dc[d][f]);
      o += 5 * (size_t)(n + 1);
    }
    FV_TRY(alloc(g, &g->d_met_fn, total * sizeof(float2)));
    FV_CUDA(cudaMemcpy(g->d_met_fn, h.data(), total * sizeof(float2), cudaMemcpyHostToDevice));
    const ffn* base = (const ffn*)g->d_met_fn;
    for (int d = 0; d < 3; ++d) {
      const int n = g->n[d];
      g->met_fn.n[d] = n;
      g->met_fn.idx[d] = base + off[d];
      g->met_fn.idc[d] = base + off[d] + (n + 1);
      g->met_fn.th[d] = base + off[d] + 2 * (n + 1);
      g->met_fn.dx[d] = base + off[d] + 3 * (n + 1);
      g->met_fn.dc[d] = base + off[d] + 4 * (n + 1);
    }
    g->met_fn.ncell = g->ncell;
    for (int d = 0; d < 3; ++d) g->met_ff.idcf[d] = (const float2*)g->met_fn.idc[d];
  }
  FV_TRY(alloc(g, (void**)&g->Uff, g->nvel * sizeof(float2)));
  FV_TRY(alloc(g, (void**)&g->xff, g->nvel * sizeof(float2)));
  FV_TRY(alloc(g, (void**)&g->d_scal, kScalars * sizeof(double)));
  FV_TRY(alloc(g, (void**)&g->d_fault, 256));
  FV_CUDA(cudaMemset(g->d_fault, 0, 256));
  g->part_len = 4096 * 130;
  FV_TRY(alloc(g, (void**)&g->d_part, g->part_len * sizeof(double)));
  FV_TRY(alloc(g, (void**)&g->wts, g->nvel * sizeof(double)));
  FV_TRY(alloc(g, (void**)&g->wts_ff, g->nvel * sizeof(float2)));
  FV_TRY(fill_face_weights(g));
  FV_CUDA(cudaMallocHost((void**)&g->h_scal, kScalars * sizeof(double)));
  FV_CUDA(cudaMemset(g->d_scal, 0, kScalars * sizeof(double)));
  return FV_OK;
}

}  // namespace fv

using namespace fv;

extern "C" {

const char* fv_last_error(void) { return g_last_error.c_str(); }

fv_status fv_grid_create(int nx, int ny, int nz, int map, double alpha, double re,
                         void* cuda_stream, fv_grid** out) {
  if (!out) { set_error("fv_grid_create: out is NULL"); return FV_EINVAL; }
  *out = nullptr;
  if (nx < 4 || ny < 4 || nz < 4 || nx > 1024 || ny > 1024 || nz > 1024) {
    set_error("fv_grid_create: each of nx, ny, nz must be in [4, 1024]");
    return FV_EINVAL;
  }
  if ((int64_t)3 * nx * ny * nz >= ((int64_t)1 << 31)) {
    set_error("fv_grid_create: 3*nx*ny*nz must be < 2^31");
    return FV_EINVAL;
  }
  if (map < 0 || map > 2) { set_error("fv_grid_create: unknown map"); return FV_EINVAL; }
  if (!(re > 0.0) || !std::isfinite(alpha)) {
    set_error("fv_grid_create: re must be > 0 and alpha finite");
    return FV_EINVAL;
  }
  fv_grid* g = new fv_grid();
  g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
  g->ncell = (int64_t)nx * ny * nz;
  g->nvel = 3 * g->ncell;
  g->map = map;
  g->alpha = alpha;
  g->re = re;
  g->stream = (cudaStream_t)cuda_stream;
  const char* ng = std::getenv("FVNS_NO_GRAPH");
  g->use_graph = !(ng && ng[0] == '1');
  fv_status s = build(g);
  if (s != FV_OK) { fv_grid_destroy(g); return s; }
  *out = g;
  return FV_OK;
}

fv_status fv_grid_set_re(fv_grid* g, double re) {
  if (!g || !(re > 0.0)) { set_error("fv_grid_set_re: bad argument"); return FV_EINVAL; }
  if (re != g->re) {
    // the captured evaluation graphs hold 1/Re as a kernel argument: drop
    // them (after the work queued on the grid's stream) so that the next
    // evaluation captures them again at the new Re
    FV_CUDA(cudaStreamSynchronize(g->stream));
    for (auto& c : g->graphs) destroy_graph_cache(c);
  }
  g->re = re;
  return FV_OK;
}

fv_status fv_grid_set_stream(fv_grid* g, void* cuda_stream) {
  if (!g) { set_error("fv_grid_set_stream: grid is NULL"); return FV_EINVAL; }
  g->stream = (cudaStream_t)cuda_stream;
  return FV_OK;
}

fv_status fv_grid_get_info(const fv_grid* g, fv_grid_info* info) {
  if (!g || !info) { set_error("fv_grid_get_info: NULL argument"); return FV_EINVAL; }
  info->nx = g->n[0]; info->ny = g->n[1]; info->nz = g->n[2];
  info->n_cell = g->ncell;
  info->n_vel = g->nvel;
  const int64_t nx = g->n[0], ny = g->n[1], nz = g->n[2];
  info->n_unknown_vel = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
  info->workspace_bytes = g->ws_bytes;
  return FV_OK;
}

fv_status fv_profile_enable(fv_grid* g, int on) {
  if (!g) { set_error("fv_profile_enable: grid is NULL"); return FV_EINVAL; }
  g->prof_on = on != 0;
  if (on) { g->ev_used = 0; g->ev_kind.clear(); }
  return FV_OK;
}

fv_status fv_profile_read(fv_grid* g, double* ms, int64_t* launches) {
  if (!g || !ms || !launches) { set_error("fv_profile_read: NULL argument"); return FV_EINVAL; }
  FV_CUDA(cudaStreamSynchronize(g->stream));
  for (int k = 0; k < FV_NKIND; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (size_t p = 0; p < g->ev_kind.size(); ++p) {
    float t = 0.f;
    FV_CUDA(cudaEventElapsedTime(&t, g->ev_pool[2 * p], g->ev_pool[2 * p + 1]));
    const int k = g->ev_kind[p];
    if (k >= 0 && k < FV_NKIND) { ms[k] += t; launches[k] += 1; }
  }
  return FV_OK;
}

int64_t fv_launch_count(void) { return g_launches.load(); }

fv_status fv_grid_set_base(fv_grid* g, const double* U) {
  if (!g || !U) { set_error("fv_grid_set_base: NULL argument"); return FV_EINVAL; }
  return set_base(g, U);
}

fv_status fv_debug_inject_status(fv_grid* g, int status) {
  if (!g) { set_error("fv_debug_inject_status: NULL grid"); return FV_EINVAL; }
  if (status != FV_ETIMEOUT) {
    set_error("fv_debug_inject_status: only FV_ETIMEOUT can be injected");
    return FV_EINVAL;
  }
  FV_CUDA(cudaMemsetAsync(g->d_fault, 0x01, 1, g->stream));
  return FV_OK;
}

void fv_grid_destroy(fv_grid* g) {
  if (!g) return;
  for (auto& c : g->graphs) destroy_graph_cache(c);
  destroy_stokes_tables(g);
  destroy_mg(g);
  if (g->d_arn) cudaFree(g->d_arn);
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  void* ptrs[] = {g->d_met_d, g->d_met_f, g->d_tpf_d, g->d_tpf_f, g->vel_buf[0], g->vel_buf[1],
                  g->vel_buf[2], g->cell_buf[0], g->cell_buf[1], g->cell_buf[2], g->tpf_buf[0],
                  g->tpf_buf[1], g->d_scal, g->d_part, g->kry, g->kry_small, g->U32, g->x32,
                  g->w32, g->vff[0], g->vff[1], g->pff, g->r32, g->phi32, g->d_met_ff,
                  g->d_met_fn, g->Uff, g->xff, g->d_tc, g->wts, g->wts_ff, g->d_fault};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (g->h_scal) cudaFreeHost(g->h_scal);
  delete g;
}

}  // extern "C"
