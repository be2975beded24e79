// One Krylov-vector evaluation (Section 3, Eqs. 8-10 and the SIMPLE-like
// loop) in the mixed precision of fv_mixed.cu, captured once per grid as a
// CUDA graph whose pass loop is a device-side WHILE conditional node:
//
//   init(call) -> base(U, if given) -> J.v -> D w -> [TPF -> correct -> decide]
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
#include <cstddef>
#include <cstring>

#include "fv_ff.cuh"
#include "fv_internal.cuh"
#include "fv_stencil_dev.cuh"
#include "fv_tc5.cuh"

namespace fv {

namespace {

// the first two members are read by the J.v kernels as their U and x
// pointers (U null: the grid's registered base flow)
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

// The evaluation's base flow when the call passes one (U non-null): rounded
// (FV_MIXED) or split (FV_FF) into the grid's stored copy that the J.v kernel
// reads; with U null the registered base flow is already there.
template <bool FF>
__global__ void k_base_from_call(const CallBlock* __restrict__ cb, float* __restrict__ U32,
                                 float2* __restrict__ Uff, int64_t n) {
  const double* U = cb->U;
  if (!U) return;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double d = __ldg(U + e);
    if (FF) {
      const ff a = f64_split(d);
      Uff[e] = make_float2(a.hi, a.lo);
    } else {
      U32[e] = f64_round_f32(d);
    }
  }
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
template <bool FIRST, bool FFG = false>
__global__ void __launch_bounds__(256) k_correct_g(MetFF m, const float* __restrict__ w32,
                                                   float2* vff0, float2* vff1,
                                                   const float* __restrict__ phi,
                                                   float2* __restrict__ p, float* __restrict__ r,
                                                   const CallBlock* __restrict__ cb,
                                                   const LoopState* __restrict__ ls,
                                                   float* __restrict__ part) {
  tc5::pdl_trigger();   // the pressure transform that follows may start its set-up
  const int done = FIRST ? 0 : ls->pass;
  // result of pass `done` is in vff[(done-1)&1]; the two buffers never overlap
  const float2* __restrict__ vin = (done & 1) ? vff0 : vff1;
  float2* __restrict__ vout = (done & 1) ? vff1 : vff0;
  const float omega = cb->omega;
  const int plane_ = m.n[0] * m.n[1];
  const int t_ = blockIdx.x * blockDim.x + threadIdx.x;
  const bool act_ = t_ < plane_;
  const int i = act_ ? t_ % m.n[0] : 0;
  const int j = act_ ? t_ / m.n[0] : 0;
  float aphi = 0.f, adiv = 0.f;
#pragma unroll
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
        if (FFG) {   // gradient of the float32 phi evaluated in float-float
          const ff gr = ff_mul(two_sum(f0, -__ldg(phi + base - st[c])), of2(m.idcf[c][q]));
          lo = ff_sub(load(c * nc + base), ff_mul_f(gr, omega));
        } else {
          const float g = (f0 - __ldg(phi + base - st[c])) * m.idc[c][q];
          lo = ff_add_f(load(c * nc + base), -omega * g);
        }
      }
      vout[c * nc + base] = to2(lo);
      if (q + 1 < m.n[c]) {
        if (FFG) {
          const ff gr = ff_mul(two_sum(__ldg(phi + base + st[c]), -f0), of2(m.idcf[c][q + 1]));
          hi = ff_sub(load(c * nc + base + st[c]), ff_mul_f(gr, omega));
        } else {
          const float g = (__ldg(phi + base + st[c]) - f0) * m.idc[c][q + 1];
          hi = ff_add_f(load(c * nc + base + st[c]), -omega * g);
        }
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
                                                 cudaGraphConditionalHandle h, int set_handle,
                                                 const unsigned* __restrict__ fault) {
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
    if (*fault) { ls->status = 4; go = 0; }   // a pressure transform's wait gave up
    else if (isinf(a) || isinf(d) || isnan(a) || isnan(d)) { ls->nan = 1; ls->status = 3; go = 0; }
    else if (a == 0.f || a <= cb->eps * phi1) { ls->status = 1; go = 0; }
    else if (pass >= 3 && a > 0.25f * prev && a <= 1e-9f * phi1) { ls->status = 1; go = 0; }
    else if (pass >= cb->max_pass) { ls->status = 2; go = 0; }
    if (set_handle) cudaGraphSetConditional(h, go ? 1u : 0u);
  }
}

__global__ void k_join_g(const float2* __restrict__ vff0, const float2* __restrict__ vff1,
                         const float2* __restrict__ pff, LoopState* __restrict__ ls,
                         const CallBlock* __restrict__ cb, int64_t nvel, int64_t ncell) {
  const float2* v = ((ls->pass - 1) & 1) ? vff1 : vff0;
  if (blockIdx.x == 0 && threadIdx.x == 0 && ls->status > ls->worst) ls->worst = ls->status;
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

}  // namespace

// Build (once per grid and shift) the executable graph of a mixed-precision
// Krylov-vector evaluation.
static_assert(offsetof(CallBlock, U) == 0 && offsetof(CallBlock, x) == sizeof(void*),
              "the J.v kernels read U and x from the head of the call block");
static fv_status build_graph(fv_grid* g, double sigma, GraphCache& gc, int prec = FV_MIXED) {
  FV_CUDA(cudaMalloc(&gc.d_call, sizeof(CallBlock)));
  FV_CUDA(cudaMalloc((void**)&gc.d_loop, sizeof(LoopState)));
  FV_CUDA(cudaMemset(gc.d_loop, 0, sizeof(LoopState)));
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
  {
    CallBlock cb0 = {};
    k_call_init<<<1, 1, 0, cs>>>(cb0, (CallBlock*)gc.d_call, gc.d_loop);
  }
  if (prec == FV_FF) {
    // float-float J.v straight from the float64 operands (or the registered
    // base flow); the predictor lands in vff[1], which the first
    // (non-initialising) pass reads, with p starting from zero
    k_base_from_call<true><<<grid1d(g->nvel), 256, 0, cs>>>(dcb, g->U32, g->Uff, g->nvel);
    if ((st = launch_jv_ff(g, nullptr, nullptr, g->vff[1], sigma, dcb)) != FV_OK) return fail(st);
    if ((st = launch_div_ff(g, g->vff[1], g->r32)) != FV_OK) return fail(st);
    if (cudaMemsetAsync(g->pff, 0, g->ncell * sizeof(float2), cs) != cudaSuccess)
      return fail(cuda_fail(cudaGetLastError(), "cudaMemsetAsync", __FILE__, __LINE__));
    if ((st = tpf_solve_f32(g, g->r32, g->phi32)) != FV_OK) return fail(st);
    k_correct_g<false, true><<<cg, bx, 0, cs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32,
                                                g->pff, g->r32, dcb, gc.d_loop, part);
  } else {
    // float32 J.v straight from the float64 operands (or the registered base)
    k_base_from_call<false><<<grid1d(g->nvel), 256, 0, cs>>>(dcb, g->U32, g->Uff, g->nvel);
    if ((st = launch_jv_f32(g, nullptr, nullptr, g->w32, sigma, dcb)) != FV_OK) return fail(st);
    if ((st = launch_div_f32(g, g->w32, g->r32)) != FV_OK) return fail(st);
    if ((st = tpf_solve_f32(g, g->r32, g->phi32)) != FV_OK) return fail(st);
    k_correct_g<true><<<cg, bx, 0, cs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32, g->pff,
                                         g->r32, dcb, gc.d_loop, part);
  }
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
  k_decide<<<1, 1024, 0, cs>>>(part, nb, gc.d_loop, dcb, h, 1, g->d_fault);
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
      if (prec == FV_FF)
        k_correct_g<false, true><<<cg, bx, 0, bs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1],
                                                    g->phi32, g->pff, g->r32, dcb, gc.d_loop, part);
      else
        k_correct_g<false><<<cg, bx, 0, bs>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32,
                                              g->pff, g->r32, dcb, gc.d_loop, part);
      k_decide<<<1, 1024, 0, bs>>>(part, nb, gc.d_loop, dcb, h, 1, g->d_fault);
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
  gc.prec = prec;
  gc.ready = true;
  return FV_OK;
}

fv_status mixed_krylov_graph(const fv_grid* gcst, const double* U, const double* x, double* out,
                             double* p, double sigma, double eps, int max_pass, double omega,
                             bool sync, int* passes, double* phi1, double* phil, double* divl,
                             int* status, int prec) {
  fv_grid* g = const_cast<fv_grid*>(gcst);
  GraphCache* gc = nullptr;
  for (auto& c : g->graphs)
    if (c.ready && c.sigma == sigma && c.prec == prec) gc = &c;
  if (!gc) {
    GraphCache* slot = nullptr;
    for (auto& c : g->graphs)
      if (!c.ready) { slot = &c; break; }
    if (!slot) slot = &g->graphs[0];
    destroy_graph_cache(*slot);
    FV_TRY(build_graph(g, sigma, *slot, prec));
    gc = slot;
  }
  CallBlock cb;
  cb.U = U;
  cb.x = x;
  if (U) g->base_ptr = nullptr;   // the graph overwrites the stored base copy
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
  if (hls.status == 4) FV_CUDA(cudaMemset(g->d_fault, 0, sizeof(unsigned)));   // reported once
  return FV_OK;
}

fv_status take_fault(const fv_grid* g, bool* hit) {
  unsigned f = 0;
  FV_CUDA(cudaMemcpyAsync(&f, g->d_fault, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
  FV_CUDA(cudaMemsetAsync(g->d_fault, 0, sizeof(unsigned), g->stream));
  FV_CUDA(cudaStreamSynchronize(g->stream));
  *hit = f != 0;
  return FV_OK;
}

fv_status status_error(int status) {
  switch (status) {
    case 2: set_error("SIMPLE loop reached max_pass"); return FV_ENOCONV;
    case 3: set_error("SIMPLE loop: NaN/Inf in the correction"); return FV_ENAN;
    case 4:
      set_error("pressure transform: a bounded wait on the tensor cores gave up (device timeout)");
      return FV_ETIMEOUT;
    default: return FV_OK;
  }
}

fv_status graph_take_status(fv_grid* g, int* worst, bool with_fault) {
  *worst = 0;
  bool hit = false;
  if (with_fault) FV_TRY(take_fault(g, &hit));
  if (hit) *worst = 4;
  for (auto& c : g->graphs) {
    if (!c.ready) continue;
    int w = 0;
    FV_CUDA(cudaMemcpyAsync(&w, &c.d_loop->worst, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
    FV_CUDA(cudaMemsetAsync(&c.d_loop->worst, 0, sizeof(int), g->stream));
    FV_CUDA(cudaStreamSynchronize(g->stream));
    *worst = std::max(*worst, w);
  }
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
      case FV_K_MOMENTUM: return launch_jv_f32(g, nullptr, g->vel_buf[1], g->w32, 0.0);
      case FV_K_DIVERGENCE: return launch_div_f32(g, g->w32, g->r32);
      case FV_K_CORRECT:
        count_launch();
        k_correct_g<false><<<cg, bx, 0, g->stream>>>(g->met_ff, g->w32, g->vff[0], g->vff[1],
                                                     g->phi32, g->pff, g->r32,
                                                     (const CallBlock*)gc->d_call, gc->d_loop, part);
        FV_CHECK_LAUNCH();
        return FV_OK;
      case FV_K_TPF_X: return tpf_one_transform_f32(g, 0);
      case FV_K_TPF_XINV: return tpf_one_transform_f32(g, 1);
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


// ===========================================================================
// Batched instances: several grids (uneven sizes, Reynolds numbers, lid
// angles) advance one Krylov-vector evaluation each in ONE graph launch.
// The momentum predictors of all instances are computed by a persistent
// work-queue kernel (blocks pull (instance, z-tile) items from an atomic
// counter, so small and large grids share the SMs); the SIMPLE loops then run
// as concurrent graph branches, one WHILE conditional node per instance.  The
// z-tile depth (planes per work item) is picked by fv_batch_autotune.
namespace {

constexpr int kBatchMax = 32;
constexpr int kBatchBlocks = 152 * 4;

struct BatchCall {
  const double* U[kBatchMax];
  const double* x[kBatchMax];
  double* out[kBatchMax];
  float eps, sigma;
  int n;
};

struct InstDesc {
  Met<float> m;
  const float* U32;
  const float* x32;
  float* w32;
  float inv_re;
  int tile_base;
};

__global__ void k_batch_init(BatchCall bc, CallBlock* dcb, LoopState* dls) {
  const int i = threadIdx.x;
  if (i >= bc.n) return;
  CallBlock c;
  c.U = bc.U[i];
  c.x = bc.x[i];
  c.out = bc.out[i];
  c.p = nullptr;
  c.sigma = bc.sigma;
  c.eps = bc.eps;
  c.omega = 1.f;
  c.max_pass = 200;
  dcb[i] = c;
  LoopState& l = dls[i];
  l.phi1 = l.phi_prev = l.phi_last = l.div_last = 0.f;
  l.pass = l.nan = l.status = 0;
}

// Momentum predictor (Eq. 10, float32) of every instance: blocks pull work
// items (instance, ppt consecutive z-planes) from an atomic counter.
__global__ void __launch_bounds__(256) k_batch_jv(const InstDesc* __restrict__ d, int ninst,
                                                  int total, int ppt, float shift,
                                                  unsigned* __restrict__ counter) {
  __shared__ int s_tile;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_tile = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int tile = s_tile;
    if (tile >= total) return;
    int inst = 0;
    while (inst + 1 < ninst && d[inst + 1].tile_base <= tile) ++inst;
    const Met<float> m = d[inst].m;
    const float* U = d[inst].U32;
    const float* V = d[inst].x32;
    float* out = d[inst].w32;
    const float inv_re = d[inst].inv_re;
    const int z0 = (tile - d[inst].tile_base) * ppt;
    const int nx = m.n[0], ny = m.n[1], nz = m.n[2];
    const int plane = nx * ny;
    const int nc = (int)m.ncell;
    const int st[3] = {1, nx, plane};
    for (int t = threadIdx.x; t < plane; t += blockDim.x) {
      const int i = t % nx, j = t / nx;
      for (int kk = 0; kk < ppt; ++kk) {
        const int k = z0 + kk;
        if (k >= nz) break;
        const int pos[3] = {i, j, k};
        const int base = k * plane + t;
        float r0 = 0.f, r1 = 0.f, r2 = 0.f;
        if (i > 0)
          r0 = stencil::momentum_face<float, 0, true, float>(m, U, V, base, pos, st, inv_re, 0.f, shift);
        if (j > 0)
          r1 = stencil::momentum_face<float, 1, true, float>(m, U, V, base, pos, st, inv_re, 0.f, shift);
        if (k > 0)
          r2 = stencil::momentum_face<float, 2, true, float>(m, U, V, base, pos, st, inv_re, 0.f, shift);
        out[base] = r0;
        out[nc + base] = r1;
        out[2 * nc + base] = r2;
      }
    }
  }
}

}  // namespace

struct BatchImpl {
  int n = 0;
  int ppt = 1;
  double sigma = 0.0;
  fv_grid* grids[kBatchMax] = {};
  cudaStream_t stream = nullptr;
  CallBlock* d_call = nullptr;
  LoopState* d_loop = nullptr;
  InstDesc* d_desc = nullptr;
  unsigned* d_counter = nullptr;
  int total_tiles = 0;
  double re[kBatchMax] = {};      // each instance's Re when the descriptors were uploaded
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraphNode_t init_node = nullptr;
  bool ready = false;
};

static fv_status batch_descriptors(BatchImpl& b) {
  std::vector<InstDesc> h(b.n);
  int base = 0;
  for (int i = 0; i < b.n; ++i) {
    fv_grid* g = b.grids[i];
    h[i].m = g->met_f;
    h[i].U32 = g->U32;
    h[i].x32 = g->x32;
    h[i].w32 = g->w32;
    h[i].inv_re = float(1.0 / g->re);
    b.re[i] = g->re;
    h[i].tile_base = base;
    base += (g->n[2] + b.ppt - 1) / b.ppt;
  }
  b.total_tiles = base;
  FV_CUDA(cudaMemcpy(b.d_desc, h.data(), b.n * sizeof(InstDesc), cudaMemcpyHostToDevice));
  return FV_OK;
}

static fv_status launch_batch_jv(BatchImpl& b, cudaStream_t s) {
  FV_CUDA(cudaMemsetAsync(b.d_counter, 0, sizeof(unsigned), s));
  const int blocks = std::min(kBatchBlocks, b.total_tiles);
  count_launch();
  k_batch_jv<<<blocks, 256, 0, s>>>(b.d_desc, b.n, b.total_tiles, b.ppt, float(b.sigma), b.d_counter);
  FV_CHECK_LAUNCH();
  return FV_OK;
}

static void batch_release_graph(BatchImpl& b) {
  if (b.exec) cudaGraphExecDestroy(b.exec);
  if (b.graph) cudaGraphDestroy(b.graph);
  b.exec = nullptr;
  b.graph = nullptr;
  b.ready = false;
}

// Capture the batch graph: init -> round (per instance) -> batched J.v ->
// per-instance branches {D w -> TPF -> correct -> decide -> WHILE{...} -> join}.
static fv_status batch_build_graph(BatchImpl& b) {
  batch_release_graph(b);
  FV_TRY(batch_descriptors(b));
  cudaStream_t cs;
  FV_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  std::vector<cudaStream_t> ss(b.n), bs(b.n);
  std::vector<cudaEvent_t> ev(b.n + 1);
  for (int i = 0; i < b.n; ++i) {
    FV_CUDA(cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking));
    FV_CUDA(cudaStreamCreateWithFlags(&bs[i], cudaStreamNonBlocking));
  }
  for (auto& e : ev) FV_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  std::vector<cudaStream_t> saved(b.n);
  for (int i = 0; i < b.n; ++i) {
    saved[i] = b.grids[i]->stream;
    b.grids[i]->capturing = true;
  }
  fv_status st = FV_OK;
  cudaGraph_t graph = nullptr;
  auto cleanup = [&]() {
    for (int i = 0; i < b.n; ++i) {
      b.grids[i]->stream = saved[i];
      b.grids[i]->capturing = false;
      cudaStreamDestroy(ss[i]);
      cudaStreamDestroy(bs[i]);
    }
    for (auto& e : ev) cudaEventDestroy(e);
    cudaStreamDestroy(cs);
  };
#define BCHK(call)                                      \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) {                            \
      st = cuda_fail(e_, #call, __FILE__, __LINE__);    \
      cudaStreamEndCapture(cs, &graph);                 \
      if (graph) cudaGraphDestroy(graph);               \
      (void)cudaGetLastError();                         \
      cleanup();                                        \
      return st;                                        \
    }                                                   \
  } while (0)
#define BTRY(call)                                      \
  do {                                                  \
    fv_status s_ = (call);                              \
    if (s_ != FV_OK) {                                  \
      cudaStreamEndCapture(cs, &graph);                 \
      if (graph) cudaGraphDestroy(graph);               \
      (void)cudaGetLastError();                         \
      cleanup();                                        \
      return s_;                                        \
    }                                                   \
  } while (0)
  BCHK(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  BatchCall bc = {};
  k_batch_init<<<1, kBatchMax, 0, cs>>>(bc, b.d_call, b.d_loop);
  BCHK(cudaGetLastError());
  for (int i = 0; i < b.n; ++i) {
    fv_grid* g = b.grids[i];
    k_round2<<<grid1d(g->nvel), 256, 0, cs>>>(b.d_call + i, g->U32, g->x32, g->nvel);
    BCHK(cudaGetLastError());
  }
  BTRY(launch_batch_jv(b, cs));
  BCHK(cudaEventRecord(ev[b.n], cs));
  for (int i = 0; i < b.n; ++i) {
    fv_grid* g = b.grids[i];
    cudaStream_t s = ss[i];
    BCHK(cudaStreamWaitEvent(s, ev[b.n], 0));
    g->stream = s;
    const int bx = kCellThreads;
    const dim3 cg = cell_launch_grid(g->n);
    const int64_t nb = (int64_t)cg.x * cg.y * cg.z;
    float* part = (float*)g->d_part;
    const CallBlock* dcb = b.d_call + i;
    LoopState* dls = b.d_loop + i;
    BTRY(launch_div_f32(g, g->w32, g->r32));
    BTRY(tpf_solve_f32(g, g->r32, g->phi32));
    k_correct_g<true><<<cg, bx, 0, s>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32, g->pff,
                                        g->r32, dcb, dls, part);
    BCHK(cudaGetLastError());
    cudaStreamCaptureStatus cst;
    cudaGraph_t cap;
    const cudaGraphNode_t* deps = nullptr;
    size_t nd = 0;
    BCHK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cap, &deps, nullptr, &nd));
    cudaGraphConditionalHandle h;
    BCHK(cudaGraphConditionalHandleCreate(&h, cap, 1, cudaGraphCondAssignDefault));
    k_decide<<<1, 1024, 0, s>>>(part, nb, dls, dcb, h, 1, g->d_fault);
    BCHK(cudaGetLastError());
    BCHK(cudaStreamGetCaptureInfo(s, &cst, nullptr, &cap, &deps, nullptr, &nd));
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    BCHK(cudaGraphAddNode(&cnode, cap, deps, nullptr, nd, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BCHK(cudaStreamBeginCaptureToGraph(bs[i], body, nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal));
    g->stream = bs[i];
    fv_status s2 = tpf_solve_f32(g, g->r32, g->phi32);
    if (s2 == FV_OK) {
      k_correct_g<false><<<cg, bx, 0, bs[i]>>>(g->met_ff, g->w32, g->vff[0], g->vff[1], g->phi32,
                                               g->pff, g->r32, dcb, dls, part);
      k_decide<<<1, 1024, 0, bs[i]>>>(part, nb, dls, dcb, h, 1, g->d_fault);
    }
    cudaGraph_t bg = body;
    cudaError_t e2 = cudaStreamEndCapture(bs[i], &bg);
    g->stream = s;
    BTRY(s2);
    BCHK(e2);
    BCHK(cudaStreamUpdateCaptureDependencies(s, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
    k_join_g<<<grid1d(g->nvel), 256, 0, s>>>(g->vff[0], g->vff[1], g->pff, dls, dcb, g->nvel,
                                             g->ncell);
    BCHK(cudaGetLastError());
    BCHK(cudaEventRecord(ev[i], s));
    BCHK(cudaStreamWaitEvent(cs, ev[i], 0));
  }
  BCHK(cudaStreamEndCapture(cs, &graph));
#undef BCHK
#undef BTRY
  cleanup();
  size_t nroot = 0;
  FV_CUDA(cudaGraphGetRootNodes(graph, nullptr, &nroot));
  std::vector<cudaGraphNode_t> roots(nroot);
  FV_CUDA(cudaGraphGetRootNodes(graph, roots.data(), &nroot));
  if (nroot != 1) {
    cudaGraphDestroy(graph);
    set_error("batch graph: unexpected root count");
    return FV_ECUDA;
  }
  b.init_node = roots[0];
  FV_CUDA(cudaGraphInstantiate(&b.exec, graph, 0));
  b.graph = graph;
  b.ready = true;
  return FV_OK;
}

}  // namespace fv

struct fv_batch {
  fv::BatchImpl impl;
};

using namespace fv;

extern "C" {

fv_status fv_batch_set_tile(fv_batch* b, int ppt);

fv_status fv_batch_create(int n, fv_grid* const* grids, void* cuda_stream, fv_batch** out) {
  if (!out || !grids || n < 1 || n > kBatchMax) {
    set_error("fv_batch_create: need 1..32 grids");
    return FV_EINVAL;
  }
  *out = nullptr;
  for (int i = 0; i < n; ++i)
    if (!grids[i]) { set_error("fv_batch_create: NULL grid"); return FV_EINVAL; }
  fv_batch* b = new fv_batch();
  BatchImpl& B = b->impl;
  B.n = n;
  for (int i = 0; i < n; ++i) B.grids[i] = grids[i];
  B.stream = (cudaStream_t)cuda_stream;
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_call, kBatchMax * sizeof(CallBlock));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_loop, kBatchMax * sizeof(LoopState));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_desc, kBatchMax * sizeof(InstDesc));
  if (e == cudaSuccess) e = cudaMalloc((void**)&B.d_counter, sizeof(unsigned));
  if (e != cudaSuccess) {
    cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
    fv_batch_destroy(b);
    return FV_ENOMEM;
  }
  *out = b;
  return FV_OK;
}

void fv_batch_destroy(fv_batch* b) {
  if (!b) return;
  BatchImpl& B = b->impl;
  batch_release_graph(B);
  void* ptrs[] = {B.d_call, B.d_loop, B.d_desc, B.d_counter};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete b;
}

fv_status fv_batch_krylov(fv_batch* b, const double* const* U, const double* const* x,
                          double* const* out, double eps, double sigma, int* passes) {
  if (!b || !U || !x || !out) { set_error("fv_batch_krylov: NULL argument"); return FV_EINVAL; }
  BatchImpl& B = b->impl;
  if (!(eps > 0) || sigma < 0) { set_error("fv_batch_krylov: bad eps/sigma"); return FV_EINVAL; }
  BatchCall bc = {};
  for (int i = 0; i < B.n; ++i) {
    if (!U[i] || !x[i] || !out[i] || x[i] == out[i]) {
      set_error("fv_batch_krylov: bad pointer");
      return FV_EINVAL;
    }
    bc.U[i] = U[i];
    bc.x[i] = x[i];
    bc.out[i] = out[i];
  }
  bc.n = B.n;
  bc.eps = (float)eps;
  bc.sigma = (float)sigma;
  if (!B.ready || B.sigma != sigma) {
    B.sigma = sigma;
    FV_TRY(batch_build_graph(B));
  } else {
    // an instance's Re changed (fv_grid_set_re): the graph reads the
    // descriptor table at run time, so uploading it again is enough
    bool stale = false;
    for (int i = 0; i < B.n; ++i) stale |= B.grids[i]->re != B.re[i];
    if (stale) {
      FV_CUDA(cudaStreamSynchronize(B.stream));
      FV_TRY(batch_descriptors(B));
    }
  }
  void* dcb = B.d_call;
  void* dls = B.d_loop;
  void* args[3] = {&bc, &dcb, &dls};
  cudaKernelNodeParams kp = {};
  kp.func = (void*)k_batch_init;
  kp.gridDim = dim3(1);
  kp.blockDim = dim3(kBatchMax);
  kp.kernelParams = args;
  FV_CUDA(cudaGraphExecKernelNodeSetParams(B.exec, B.init_node, &kp));
  // the batch rounds each instance's U into the grid's U32, replacing a
  // base flow registered on that grid
  for (int i = 0; i < B.n; ++i) B.grids[i]->base_ptr = nullptr;
  count_launch();
  FV_CUDA(cudaGraphLaunch(B.exec, B.stream));
  if (passes) {
    std::vector<LoopState> h(B.n);
    FV_CUDA(cudaMemcpyAsync(h.data(), B.d_loop, B.n * sizeof(LoopState), cudaMemcpyDeviceToHost,
                            B.stream));
    FV_CUDA(cudaStreamSynchronize(B.stream));
    for (int i = 0; i < B.n; ++i) passes[i] = h[i].pass;
    int worst = 1;
    for (int i = 0; i < B.n; ++i) {
      if (h[i].status == 4) FV_CUDA(cudaMemsetAsync(B.grids[i]->d_fault, 0, sizeof(unsigned), B.stream));
      worst = std::max(worst, h[i].status == 0 ? 2 : h[i].status);
    }
    if (worst != 1) {
      const fv_status e = status_error(worst);
      set_error(std::string("fv_batch_krylov: an instance did not converge: ") + fv_last_error());
      return e;
    }
  }
  return FV_OK;
}

fv_status fv_batch_autotune(fv_batch* b, int* best_ppt, double* ms) {
  if (!b || !best_ppt) { set_error("fv_batch_autotune: NULL argument"); return FV_EINVAL; }
  BatchImpl& B = b->impl;
  static const int cand[4] = {1, 2, 4, 8};
  cudaEvent_t e0, e1;
  FV_CUDA(cudaEventCreate(&e0));
  FV_CUDA(cudaEventCreate(&e1));
  double best = 1e30;
  int bp = 1;
  for (int c = 0; c < 4; ++c) {
    B.ppt = cand[c];
    FV_TRY(batch_descriptors(B));
    FV_TRY(launch_batch_jv(B, B.stream));          // warm-up
    FV_CUDA(cudaEventRecord(e0, B.stream));
    for (int r = 0; r < 10; ++r) FV_TRY(launch_batch_jv(B, B.stream));
    FV_CUDA(cudaEventRecord(e1, B.stream));
    FV_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    FV_CUDA(cudaEventElapsedTime(&t, e0, e1));
    if (ms) ms[c] = t / 10.0;
    if (t < best) { best = t; bp = cand[c]; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ppt = bp;
  B.ppt = 0;                                       // force the graph rebuild below
  return fv_batch_set_tile(b, bp);
}

fv_status fv_batch_set_tile(fv_batch* b, int ppt) {
  if (!b || ppt < 1 || ppt > 64) { set_error("fv_batch_set_tile: bad argument"); return FV_EINVAL; }
  BatchImpl& B = b->impl;
  if (B.ppt != ppt) {
    B.ppt = ppt;
    batch_release_graph(B);
  }
  return FV_OK;
}

}  // extern "C"

extern "C" fv_status fv_bench_kernel(fv_grid* g, int kind, int reps, double* ms_per_launch) {
  if (!g || !ms_per_launch || reps < 1) { fv::set_error("fv_bench_kernel: bad argument"); return FV_EINVAL; }
  return fv::bench_kernel(g, kind, reps, ms_per_launch);
}
