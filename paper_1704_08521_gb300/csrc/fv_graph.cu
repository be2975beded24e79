// One Krylov-vector evaluation (Section 3, Eqs. 8-10 and the SIMPLE-like
// loop) in the mixed precision of fv_mixed.cu, captured once per grid as a
// CUDA graph whose pass loop is a device-side WHILE conditional node:
//
//   init(call) -> round(U, x) -> J.v -> D w -> [TPF -> correct -> decide]
//   -> while (decide says go on) { TPF -> correct -> decide } -> join
//
// The stop test of the loop (||phi_k|| <= eps ||phi_1||, round-off floor,
// pass cap) is taken on the device by the one-block `decide` kernel, so a
// whole evaluation is one graph launch with no host round trip.  Per-call
// arguments (pointers, eps, omega) are kernel arguments of the first node,
// updated in the executable graph before each launch; the loop reads them
// from a small device block.  The velocity state alternates between two
// float-float buffers by pass parity, read from the loop state.
#include <algorithm>
#include <cstring>

#include "fv_ff.cuh"
#include "fv_internal.cuh"

namespace fv {

namespace {

struct CallBlock {
  const double* U;
  const double* x;
  double* out;
  double* p;
  float sigma, eps, omega;
  int max_pass;
};

__device__ __forceinline__ float2 to2(ff a) { return make_float2(a.hi, a.lo); }
__device__ __forceinline__ ff of2(float2 a) { return {a.x, a.y}; }

__global__ void k_call_init(CallBlock cb, CallBlock* dcb, LoopState* ls) {
  *dcb = cb;
  ls->phi1 = ls->phi_prev = ls->phi_last = ls->div_last = 0.f;
  ls->pass = 0;
  ls->nan = 0;
  ls->status = 0;
}

__global__ void k_round2(const CallBlock* __restrict__ cb, float* __restrict__ U32,
                         float* __restrict__ x32, int64_t n) {
  const double* U = cb->U;
  const double* x = cb->x;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    U32[e] = f64_round_f32(__ldg(U + e));
    x32[e] = f64_round_f32(__ldg(x + e));
  }
}

__device__ __forceinline__ float block_maxf(float v) {
  __shared__ float red[32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = (lane < nw) ? red[lane] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  return v;
}

// One SIMPLE pass on the float-float state (see k_correct_ff in
// fv_mixed.cu); buffers chosen by the number of completed passes.  Block
// maxima of |phi| and |D v| go to per-block partials (no atomics).
template <bool FIRST>
__global__ void __launch_bounds__(256) k_correct_g(MetFF m, const float* __restrict__ w32,
                                                   float2* vff0, float2* vff1,
                                                   const float* __restrict__ phi,
                                                   float2* __restrict__ p, float* __restrict__ r,
                                                   const CallBlock* __restrict__ cb,
                                                   const LoopState* __restrict__ ls,
                                                   float* __restrict__ part) {
  const int done = FIRST ? 0 : ls->pass;
  const float2* vin = (done & 1) ? vff0 : vff1;   // result of pass `done` is in vff[(done-1)&1]
  float2* vout = (done & 1) ? vff1 : vff0;
  const float omega = cb->omega;
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  float aphi = 0.f, adiv = 0.f;
  for (int kk = 0; kk < kCellKz; ++kk) {
    const int k = blockIdx.y * kCellKz + kk;
    if (!act_ || k >= m.n[2]) continue;
    const int pos[3] = {i, j, k};
    const int st[3] = {1, m.n[0], m.n[0] * m.n[1]};
    const int nc = (int)m.ncell;
    const int base = (k * m.n[1] + j) * m.n[0] + i;
    auto load = [&](int e) -> ff {
      if (FIRST) return {__ldg(w32 + e), 0.f};
      return of2(vin[e]);
    };
    const float f0 = __ldg(phi + base);
    ff dv = {0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = pos[c];
      ff lo = {0.f, 0.f}, hi = {0.f, 0.f};
      if (q > 0) {
        const float g = (f0 - __ldg(phi + base - st[c])) * m.idc[c][q];
        lo = ff_add_f(load(c * nc + base), -omega * g);
      }
      vout[c * nc + base] = to2(lo);
      if (q + 1 < m.n[c]) {
        const float g = (__ldg(phi + base + st[c]) - f0) * m.idc[c][q + 1];
        hi = ff_add_f(load(c * nc + base + st[c]), -omega * g);
      }
      dv = ff_add(dv, ff_mul(ff_sub(hi, lo), of2(m.idx[c][q])));
    }
    r[base] = dv.hi;
    if (FIRST) p[base] = make_float2(omega * f0, 0.f);
    else p[base] = to2(ff_add_f(of2(p[base]), omega * f0));
    float a1 = fabsf(f0), a2 = fabsf(dv.hi);
    if (!(a1 <= 3e38f) || !(a2 <= 3e38f)) a1 = a2 = __int_as_float(0x7f800000);
    aphi = fmaxf(aphi, a1);
    adiv = fmaxf(adiv, a2);
  }
  aphi = block_maxf(aphi);
  adiv = block_maxf(adiv);
  if (threadIdx.x == 0) {
    const int64_t b = ((int64_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    const int64_t nb = (int64_t)gridDim.x * gridDim.y * gridDim.z;
    part[b] = aphi;
    part[nb + b] = adiv;
  }
}

// Stop test of the SIMPLE loop (Section 3: until ||phi|| < eps, read as
// ||phi_k||_inf <= eps ||phi_1||_inf; plus the round-off floor and the pass
// cap).  Sets the WHILE condition of the graph.
__global__ void __launch_bounds__(1024) k_decide(const float* __restrict__ part, int64_t nb,
                                                 LoopState* ls, const CallBlock* __restrict__ cb,
                                                 cudaGraphConditionalHandle h, int set_handle) {
  float a = 0.f, d = 0.f;
  for (int64_t b = threadIdx.x; b < nb; b += blockDim.x) {
    a = fmaxf(a, part[b]);
    d = fmaxf(d, part[nb + b]);
  }
  a = block_maxf(a);
  d = block_maxf(d);
  if (threadIdx.x == 0) {
    const int pass = ls->pass + 1;
    ls->pass = pass;
    if (pass == 1) ls->phi1 = a;
    const float prev = ls->phi_last;
    ls->phi_prev = prev;
    ls->phi_last = a;
    ls->div_last = d;
    const float phi1 = ls->phi1;
    int go = 1;
    if (isinf(a) || isinf(d) || isnan(a) || isnan(d)) { ls->nan = 1; ls->status = 3; go = 0; }
    else if (a == 0.f || a <= cb->eps * phi1) { ls->status = 1; go = 0; }
    else if (pass >= 3 && a > 0.25f * prev && a <= 1e-9f * phi1) { ls->status = 1; go = 0; }
    else if (pass >= cb->max_pass) { ls->status = 2; go = 0; }
    if (set_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

__global__ void k_join_g(const float2* __restrict__ vff0, const float2* __restrict__ vff1,
                         const float2* __restrict__ pff, const LoopState* __restrict__ ls,
                         const CallBlock* __restrict__ cb, int64_t nvel, int64_t ncell) {
  const float2* v = ((ls->pass - 1) & 1) ? vff1 : vff0;
  const double* x = cb->x;
  double* out = cb->out;
  double* p = cb->p;
  const float sigma = cb->sigma;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nvel;
       e += (int64_t)gridDim.x * blockDim.x) {
    ff a = of2(v[e]);
    if (sigma != 0.f) a = ff_sub(a, ff_mul_f(f64_split(__ldg(x + e)), sigma));
    out[e] = ff_join(a.hi, a.lo);
    if (p && e < ncell) {
      const ff q = of2(pff[e]);
      p[e] = ff_join(q.hi, q.lo);
    }
  }
}

inline unsigned grid1d(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  return (unsigned)(b < 1 ? 1 : b);
}

inline int block_x(const fv_grid*) { return kCellThreads; }

// Record the evaluation on stream s (capturing); `h` valid when in the body.
fv_status record_prefix(const fv_grid* g, cudaStream_t s, double sigma, GraphCache& gc) {
  const int bx = block_x(g);
  const dim3 cg = cell_launch_grid(g->n);
  CallBlock cb = {};
  k_call_init<<<1, 1, 0, s>>>(cb, (CallBlock*)gc.d_call, gc.d_loop);
  FV_CHECK_LAUNCH();
  k_round2<<<grid1d(g->nvel), 256, 0, s>>>((const CallBlock*)gc.d_call, g->U32, g->x32, g->nvel);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

}  // namespace

// Build (once per grid and shift) the executable graph of a mixed-precision
// Krylov-vector evaluation.
static fv_status build_graph(fv_grid* g, double sigma, GraphCache& gc) {
  FV_CUDA(cudaMalloc(&gc.d_call, sizeof(CallBlock)));
  FV_CUDA(cudaMalloc((void**)&gc.d_loop, sizeof(LoopState)));
  cudaStream_t cs;
  FV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  const cudaStream_t saved = g->stream;
  g->stream = cs;                     // the launch helpers enqueue on g->stream
  const bool prof = g->prof_on;
  g->prof_on = false;
  g->capturing = true;
  fv_status st = FV_OK;
  cudaGraph_t graph = nullptr;
  auto fail = [&](fv_status s) {
    cudaStreamEndCapture(cs, &graph);
    if (graph) cudaGraphDestroy(graph);
    (void)cudaGetLastError();
    g->stream = saved;
    g->prof_on = prof;
    g->capturing = false;
    cudaStreamDestroy(cs);
    return s;
  };
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaStreamBeginCapture", __FILE__, __LINE__));
  const int bx = block_x(g);
  const dim3 cg = cell_launch_grid(g->n);
  const int64_t nb = (int64_t)cg.x * cg.y * cg.z;
  float* part = (float*)g->d_part;
  const CallBlock* dcb = (const CallBlock*)gc.d_call;
  if ((st = record_prefix(g, cs, sigma, gc)) != FV_OK) return fail(st);
  if ((st = launch_momentum_f32(g, g->U32, g->x32, g->w32, sigma)) != FV_OK) return fail(st);
  if ((st = launch_div_f32(g, g->w32, g->r32)) != FV_OK) return fail(st);
  if ((st = tpf_solve_f32(g, g->r32, g->phi32)) != FV_OK) return fail(st);
  k_correct_g<true><<<cg, bx, 0, cs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32, g->pff,
                                       g->r32, dcb, gc.d_loop, part);
  // the conditional handle belongs to the graph being captured
  cudaStreamCaptureStatus cst;
  cudaGraph_t cap_graph;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap_graph, &deps, nullptr, &ndeps) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaStreamGetCaptureInfo", __FILE__, __LINE__));
  cudaGraphConditionalHandle h;
  if (cudaGraphConditionalHandleCreate(&h, cap_graph, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaGraphConditionalHandleCreate", __FILE__, __LINE__));
  k_decide<<<1, 1024, 0, cs>>>(part, nb, gc.d_loop, dcb, h, 1);
  if (cudaStreamGetCaptureInfo(cs, &cst, nullptr, &cap_graph, &deps, nullptr, &ndeps) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaStreamGetCaptureInfo", __FILE__, __LINE__));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  if (cudaGraphAddNode(&cnode, cap_graph, deps, nullptr, ndeps, &cp) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaGraphAddNode(conditional)", __FILE__, __LINE__));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  {
    cudaStream_t bs;
    if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess)
      return fail(cuda_fail(cudaGetLastError(), "cudaStreamCreate", __FILE__, __LINE__));
    if (cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(bs);
      return fail(cuda_fail(cudaGetLastError(), "cudaStreamBeginCaptureToGraph", __FILE__, __LINE__));
    }
    g->stream = bs;
    fv_status s2 = tpf_solve_f32(g, g->r32, g->phi32);
    if (s2 == FV_OK) {
      k_correct_g<false><<<cg, bx, 0, bs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32,
                                            g->pff, g->r32, dcb, gc.d_loop, part);
      k_decide<<<1, 1024, 0, bs>>>(part, nb, gc.d_loop, dcb, h, 1);
    }
    cudaGraph_t bg = body;
    cudaError_t e2 = cudaStreamEndCapture(bs, &bg);
    cudaStreamDestroy(bs);
    g->stream = cs;
    if (s2 != FV_OK) return fail(s2);
    if (e2 != cudaSuccess) return fail(cuda_fail(e2, "cudaStreamEndCapture(body)", __FILE__, __LINE__));
  }
  if (cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaStreamUpdateCaptureDependencies", __FILE__, __LINE__));
  k_join_g<<<grid1d(g->nvel), 256, 0, cs>>>(g->vff[0], g->vff[1], g->pff, gc.d_loop, dcb, g->nvel,
                                            g->ncell);
  if (cudaStreamEndCapture(cs, &graph) != cudaSuccess)
    return fail(cuda_fail(cudaGetLastError(), "cudaStreamEndCapture", __FILE__, __LINE__));
  g->stream = saved;
  g->prof_on = prof;
  g->capturing = false;
  cudaStreamDestroy(cs);
  // the first node (k_call_init) carries the per-call arguments
  size_t nroot = 0;
  FV_CUDA(cudaGraphGetRootNodes(graph, nullptr, &nroot));
  std::vector<cudaGraphNode_t> roots(nroot);
  FV_CUDA(cudaGraphGetRootNodes(graph, roots.data(), &nroot));
  if (nroot != 1) { cudaGraphDestroy(graph); set_error("graph: unexpected root count"); return FV_ECUDA; }
  gc.init_node = roots[0];
  FV_CUDA(cudaGraphInstantiate(&gc.exec, graph, 0));
  gc.graph = graph;
  gc.sigma = sigma;
  gc.ready = true;
  return FV_OK;
}

fv_status mixed_krylov_graph(const fv_grid* gcst, const double* U, const double* x, double* out,
                             double* p, double sigma, double eps, int max_pass, double omega,
                             bool sync, int* passes, double* phi1, double* phil, double* divl,
                             int* status) {
  fv_grid* g = const_cast<fv_grid*>(gcst);
  GraphCache* gc = nullptr;
  for (auto& c : g->graphs)
    if (c.ready && c.sigma == sigma) gc = &c;
  if (!gc) {
    GraphCache* slot = nullptr;
    for (auto& c : g->graphs)
      if (!c.ready) { slot = &c; break; }
    if (!slot) slot = &g->graphs[0];
    destroy_graph_cache(*slot);
    FV_TRY(build_graph(g, sigma, *slot));
    gc = slot;
  }
  CallBlock cb;
  cb.U = U;
  cb.x = x;
  cb.out = out;
  cb.p = p;
  cb.sigma = (float)sigma;
  cb.eps = (float)eps;
  cb.omega = (float)omega;
  cb.max_pass = max_pass;
  void* dcb = gc->d_call;
  LoopState* dls = gc->d_loop;
  void* args[3] = {&cb, &dcb, &dls};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_call_init;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(1);
  kp.sharedMemBytes = 0;
  kp.kernelParams = args;
  FV_CUDA(cudaGraphExecKernelNodeSetParams(gc->exec, gc->init_node, &kp));
  count_launch();                     // one graph launch
  FV_CUDA(cudaGraphLaunch(gc->exec, g->stream));
  if (!sync) return FV_OK;
  LoopState hls;
  FV_CUDA(cudaMemcpyAsync(&hls, dls, sizeof(LoopState), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  if (passes) *passes = hls.pass;
  if (phi1) *phi1 = hls.phi1;
  if (phil) *phil = hls.phi_last;
  if (divl) *divl = hls.div_last;
  if (status) *status = hls.status;
  return FV_OK;
}

// Back-to-back launches of one kernel class of the mixed path on the grid's
// current workspace (left by a previous evaluation), timed with CUDA events on
// the grid's stream: average device time per launch.
fv_status bench_kernel(fv_grid* g, int kind, int reps, double* ms) {
  GraphCache* gc = nullptr;
  for (auto& c : g->graphs)
    if (c.ready) gc = &c;
  if (!gc) {
    // host-driven grids have no graph yet: capture one for its device blocks
    gc = &g->graphs[0];
    FV_TRY(build_graph(g, 0.0, *gc));
    FV_CUDA(cudaMemsetAsync(gc->d_call, 0, sizeof(CallBlock), g->stream));
    FV_CUDA(cudaMemsetAsync(gc->d_loop, 0, sizeof(LoopState), g->stream));
  }
  const int bx = block_x(g);
  const dim3 cg = cell_launch_grid(g->n);
  float* part = (float*)g->d_part;
  cudaEvent_t e0, e1;
  FV_CUDA(cudaEventCreate(&e0));
  FV_CUDA(cudaEventCreate(&e1));
  auto one = [&]() -> fv_status {
    switch (kind) {
      case FV_K_MOMENTUM: return launch_momentum_f32(g, g->U32, g->x32, g->w32, 0.0);
      case FV_K_DIVERGENCE: return launch_div_f32(g, g->w32, g->r32);
      case FV_K_CORRECT:
        count_launch();
        k_correct_g<false><<<cg, bx, 0, g->stream>>>(g->met_ff, g->w32, g->vff[0], g->vff[1],
                                                     g->phi32, g->pff, g->r32,
                                                     (const CallBlock*)gc->d_call, gc->d_loop, part);
        FV_CHECK_LAUNCH();
        return FV_OK;
      case FV_K_TPF_X: return tpf_one_transform_f32(g, 0);
      case FV_K_TPF_YZ: return tpf_one_transform_f32(g, 2);
      default: set_error("fv_bench_kernel: unsupported kind"); return FV_EINVAL;
    }
  };
  FV_TRY(one());                                   // warm-up
  FV_CUDA(cudaEventRecord(e0, g->stream));
  for (int r = 0; r < reps; ++r) FV_TRY(one());
  FV_CUDA(cudaEventRecord(e1, g->stream));
  FV_CUDA(cudaEventSynchronize(e1));
  float t = 0.f;
  FV_CUDA(cudaEventElapsedTime(&t, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t / reps;
  return FV_OK;
}

void destroy_graph_cache(GraphCache& c) {
  if (c.exec) cudaGraphExecDestroy(c.exec);
  if (c.graph) cudaGraphDestroy(c.graph);
  if (c.d_call) cudaFree(c.d_call);
  if (c.d_loop) cudaFree(c.d_loop);
  c = GraphCache();
}

}  // namespace fv

extern "C" fv_status fv_bench_kernel(fv_grid* g, int kind, int reps, double* ms_per_launch) {
  if (!g || !ms_per_launch || reps < 1) { fv::set_error("fv_bench_kernel: bad argument"); return FV_EINVAL; }
  return fv::bench_kernel(g, kind, reps, ms_per_launch);
}
