// Launch sequences of the single-instance HPR-QP solver and the CUDA graphs that run them.
//
// Fixed-schedule graph (one launch = L inner steps, L = lcm(restart_every, check_every)):
//   dispatch -> step 1 -> ... -> step L, the variant of each step fixed by its position (R~
// test at multiples of restart_every, stopping test at multiples of check_every); the step
// after each R~ test is a SWITCH node (scheduled step / step with R~_{r,0} after a restart
// without sigma update / restart pass of Algorithm 5 then that step / nothing once done).
// Dynamic graph (one launch = iters_per_launch steps, for the iterations after the last whole
// period):
//   dispatch -> [SWITCH step 0] -> [IF restart 0] -> [SWITCH step 1] -> [IF restart 1] -> ...
// each SWITCH with four bodies: plain step, step with the R~ test (Sec. 3.2), step with the
// stopping rule (Sec. 4.1), empty once done.  In both, the controller in the last block of
// every step sets the next conditional node with cudaGraphSetConditional, so the host only
// polls a done flag between launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <utility>
#include <vector>

#include "kernels.cuh"

namespace hprqp {

static RowKernel rowk(int kind, int var, int G) {
  if (kind == K_Q1 || kind == K_Q2 || kind == K_APPLY_Q || kind == K_POWER_Q || kind == K_Q2H)
    return row_kernel_q(kind, var, G);
  if (kind == K_A1 || kind == K_APPLY_A || kind == K_POWER_A) return row_kernel_a(kind, var, G);
  return row_kernel_at(kind, var, G);
}

using PreKernel = void (*)(Args, int);
static PreKernel prek(int G, int tt) {
#define HPRQP_PRE(GG) \
  case GG:            \
    return tt == 0 ? k_pre<GG, 0> : tt == 1 ? k_pre<GG, 1> : k_pre<GG, 2>;
  switch (G) {
    HPRQP_PRE(1)
    HPRQP_PRE(4)
    HPRQP_PRE(8)
    default:
      return tt == 0 ? k_pre<32, 0> : tt == 1 ? k_pre<32, 1> : k_pre<32, 2>;
  }
#undef HPRQP_PRE
}

using ZxKernel = void (*)(Args);
static ZxKernel zxk(int var) {
  switch (var) {
    case VAR_PLAIN: return k_zx<VAR_PLAIN>;
    case VAR_R: return k_zx<VAR_R>;
    case VAR_T: return k_zx<VAR_T>;
    default: return k_zx<VAR_RUNTIME>;
  }
}

// Optional per-kind timing: ev[kind][0/1] recorded around every launch of that kind.
#define TIMED(kind, launch)                  \
  do {                                       \
    if (ev) cudaEventRecord(ev[kind][0], s); \
    launch;                                  \
    if (ev) cudaEventRecord(ev[kind][1], s); \
  } while (0)


// ------------------------------------------------------------------------------------ QAP term
__global__ void k_qap_diff(const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ out,
                           int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = a[i] - b[i];
}

cudaError_t launch_qap(const Args& a, const Plan& p, int which, int tt, cudaStream_t s) {
  const QDev& Q = a.Q;
  if (!Q.qap_d) return cudaSuccess;
  const Vec& V = a.V;
  double* t = pre_into_t1(which) ? V.t1 : V.t2;
  const double* x = which == PRE_WH ? (a.m > 0 ? V.wh : V.wb) : which == PRE_WB ? V.wb : which == PRE_AIN ? V.ain
                    : which == PRE_PV ? V.pv : which == PRE_W ? V.w : Q.qap_in;
  if (which == 2) {
    const int blocks = (int)std::min<int64_t>((a.n + kThreads - 1) / kThreads, 152 * 8);
    k_qap_diff<<<blocks, kThreads, 0, s>>>(V.ATyb, V.ATy0, Q.qap_in, a.n);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = qap_apply(Q, x, t + Q.qap_off, Q.qap_splits, s);
  if (e == cudaSuccess && which == 0 && tt != 0) e = qap_apply(Q, V.xb, t + Q.tlen + Q.qap_off, Q.qap_splits, s);
  return e;
}

// Launches kernel k; with pdl set it is a programmatic dependent launch (it may start while
// the previous kernel of the stream drains; the kernel itself waits for that kernel's results).
template <typename... P, typename... A>
static cudaError_t launch_k(bool pdl, void (*k)(P...), int grid, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  return cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

// Kernel sequence on one stream: programmatic launches only directly after another kernel of
// this library (not first in a graph body, not after cuBLAS, not between profiling events).
struct Seq {
  cudaStream_t s;
  bool pdl;
  bool prev = false;
  cudaError_t e = cudaSuccess;
  int count = 0;   // kernels launched through this sequence
  template <typename... P, typename... A>
  void operator()(void (*k)(P...), int grid, A&&... args) {
    if (e == cudaSuccess) e = launch_k(pdl && prev, k, grid, s, std::forward<A>(args)...);
    prev = true;
    count++;
  }
  void other() { prev = false; }
};

// Whether the CSR pre-pass has work before a Q pass: dense factors, factors without a tiled
// copy, or the two-vector pass of a stopping test (tiled factors take the CSR path there).
static bool pre_has_work(const Args& a, int which, int tt) {
  if (!a.Q.has_fd()) return false;
  if (a.Q.ndense) return true;
  const bool step = which == PRE_WH || which == PRE_WB || which == PRE_W || which == PRE_PV;
  bool tiled = false;
  for (int f = 0; f < a.Q.nfac; f++) {
    if (!a.Q.tiled[f] && !(step && a.Q.inl[f])) return true;
    tiled = tiled || a.Q.tiled[f];
  }
  return which == PRE_WH && tt != 0 && tiled;
}
static int tiled_terms(const Args& a) {
  int c = 0;
  for (int f = 0; f < a.Q.nfac; f++) c += a.Q.tiled[f];
  return c;
}

// Shape of an inner step in the fixed-schedule graph.  k1: the step begins with its own k_zx
// (false when the step before ran it in K_Q2H); fuse_next >= 0 (plain steps only): the step
// ends with K_ATH and K_Q2H, which run the elementwise pass of the next step, a step of variant
// fuse_next; k1_after >= 0: the step ends with the next step's k_zx in that variant.
struct StepShape {
  bool k1 = true;
  int fuse_next = -1;
  int k1_after = -1;
  int* kernels = nullptr;   // optional: receives += the number of kernels the step launches
};

// One inner step in variant `var`; the last kernel of the step receives the handles.  chained:
// the previous node on s is this library's kernel (its first kernel may then launch early too).
cudaError_t launch_step(const Args& a, const Plan& p, cudaStream_t s, int var, const Handles& hd,
                        cudaEvent_t (*ev)[2], bool chained = false, StepShape sh = StepShape()) {
  const bool HQ = a.Q.present(), HA = a.m > 0, pre = a.Q.has_pre();
  const Handles none;
  const int tt = var == VAR_T ? 1 : var == VAR_RUNTIME ? 2 : 0;
  // plain steps write no partial sums, so they may run at their own (larger) grids
  const bool pl = var == VAR_PLAIN && p.wZX > 0;
  Seq L{s, p.pdl != 0 && !ev};
  L.prev = chained;
  // the products that precede a Q pass: CSR pre-pass, tiled factor kernels, QAP contractions
  auto pre_pass = [&](int which, int ptt) -> cudaError_t {
    if (pre_has_work(a, which, ptt)) L(prek(p.gPre, ptt), p.gridPre, a, which);
    if (L.e != cudaSuccess) return L.e;
    if (tiled_terms(a)) {
      int nt = 0;
      const cudaError_t te = launch_tiled(a, p, which, ptt, s, &nt);
      if (te != cudaSuccess) return te;
      if (nt) L.prev = true;
      L.count += nt;
    }
    if (a.Q.qap_d) {
      L.other();
      const cudaError_t qe = launch_qap(a, p, which, ptt, s);
      if (qe != cudaSuccess) return qe;
      L.count += 2 + (which == PRE_WH && ptt != 0 ? 2 : 0);
    }
    return cudaSuccess;
  };
  const bool fused = sh.fuse_next >= 0 && var == VAR_PLAIN && HQ && HA;
  if (sh.k1) TIMED(0, L(zxk(var), pl ? p.wZX : p.gridE, a));
  if (HQ) {
    if (pre) {
      if (ev) cudaEventRecord(ev[1][0], s);
      const cudaError_t pe = pre_pass(0, tt);
      if (pe != cudaSuccess) return pe;
      if (ev) cudaEventRecord(ev[1][1], s);
    }
    TIMED(2, L(rowk(K_Q1, var, p.gQ), pl ? p.wQ1 : p.gridN, a, HA ? none : hd));
  }
  if (HA) {
    TIMED(3, L(rowk(K_A1, var, p.gA), pl ? p.wA1 : p.gridM, a, none));
    if (fused) {
      TIMED(9, L(rowk(K_ATH, VAR_PLAIN, p.gAT), p.wATH, a, none));
      if (pre) {
        if (ev) cudaEventRecord(ev[10][0], s);
        const cudaError_t pe = pre_pass(PRE_W, 0);
        if (pe != cudaSuccess) return pe;
        if (ev) cudaEventRecord(ev[10][1], s);
      }
      TIMED(11, L(rowk(K_Q2H, sh.fuse_next, p.gQ), p.wQ2H, a, hd));
      if (sh.kernels) *sh.kernels += L.count;
      if (L.e != cudaSuccess) return L.e;
      return cudaGetLastError();
    }
    TIMED(4, L(rowk(K_AT, var, p.gAT), pl ? p.wAT : p.gridN, a, HQ ? none : hd));
    if (HQ) {
      if (pre) {
        if (ev) cudaEventRecord(ev[5][0], s);
        const cudaError_t pe = pre_pass(1, 0);
        if (pe != cudaSuccess) return pe;
        if (ev) cudaEventRecord(ev[5][1], s);
      }
      TIMED(6, L(rowk(K_Q2, var, p.gQ), pl ? p.wQ2 : p.gridN, a, hd));
    }
  }
  if (!HQ && !HA) {
    // neither operator: the controller still needs its (empty-operator) pass
    TIMED(4, L(rowk(K_AT, var, p.gAT), p.gridN, a, hd));
  }
  if (sh.k1_after >= 0) L(zxk(sh.k1_after), sh.k1_after == VAR_PLAIN && p.wZX > 0 ? p.wZX : p.gridE, a);
  if (sh.kernels) *sh.kernels += L.count;
  if (L.e != cudaSuccess) return L.e;
  return cudaGetLastError();
}

__global__ void k_vmul(double* __restrict__ out, const double* __restrict__ v, const double* __restrict__ sc,
                       int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += stride) out[i] = v[i] * sc[i];
}

cudaError_t launch_vmul_to(double* out, const double* v, const double* sc, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int blocks = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
  k_vmul<<<blocks, kThreads, 0, st>>>(out, v, sc, n);
  return cudaGetLastError();
}

cudaError_t launch_vmul(double* v, const double* sc, int64_t n, cudaStream_t st) {
  return launch_vmul_to(v, v, sc, n, st);
}

__global__ void k_stamp(Ctrl* C) {
  if (threadIdx.x == 0 && blockIdx.x == 0) C->t0_ns = global_ns();
}

cudaError_t launch_stamp(const Args& a, cudaStream_t s) {
  k_stamp<<<1, 32, 0, s>>>(a.C);
  return cudaGetLastError();
}

cudaError_t plan_plain_grids(const Args& a, Plan& p, int sms) {
  auto wave = [sms](const void* f, int64_t units) -> int {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kThreads, 0) != cudaSuccess || occ < 1) occ = 1;
    const int64_t need = std::max<int64_t>(1, units);
    return (int)std::min<int64_t>(need, (int64_t)sms * occ);
  };
  const int64_t chN = (a.n + kChunk - 1) / kChunk, chM = (a.m + kChunk - 1) / kChunk;
  p.wZX = wave((const void*)zxk(VAR_PLAIN), (a.n + kThreads - 1) / kThreads);
  p.wQ1 = wave((const void*)rowk(K_Q1, VAR_PLAIN, p.gQ), chN);
  p.wQ2 = wave((const void*)rowk(K_Q2, VAR_PLAIN, p.gQ), chN);
  p.wAT = wave((const void*)rowk(K_AT, VAR_PLAIN, p.gAT), chN);
  p.wA1 = wave((const void*)rowk(K_A1, VAR_PLAIN, p.gA), std::max<int64_t>(chM, 1));
  p.wATH = wave((const void*)rowk(K_ATH, VAR_PLAIN, p.gAT), chN);
  p.wQ2H = wave((const void*)rowk(K_Q2H, VAR_PLAIN, p.gQ), chN);
  return cudaGetLastError();
}

cudaError_t launch_restart(const Args& a, const Plan& p, cudaStream_t s, cudaEvent_t (*ev)[2]) {
  Seq L{s, p.pdl != 0 && !ev};
  if (a.Q.present() && a.m > 0 && a.Q.has_pre()) {
    if (ev) cudaEventRecord(ev[7][0], s);
    if (pre_has_work(a, 2, 0)) L(prek(p.gPre, 0), p.gridPre, a, 2);
    if (tiled_terms(a)) {
      int nt = 0;
      const cudaError_t te = launch_tiled(a, p, 2, 0, s, &nt);
      if (te != cudaSuccess) return te;
      if (nt) L.prev = true;
    }
    if (a.Q.qap_d) {
      L.other();
      const cudaError_t qe = launch_qap(a, p, 2, 0, s);
      if (qe != cudaSuccess) return qe;
    }
    if (ev) cudaEventRecord(ev[7][1], s);
  }
  const int G = p.gQ;
  void (*kr)(Args) = G <= 1 ? k_restart<1> : G == 2 ? k_restart<2> : G == 4 ? k_restart<4>
                     : G == 8 ? k_restart<8> : G == 16 ? k_restart<16> : k_restart<32>;
  TIMED(8, L(kr, p.gridN, a));
  if (L.e != cudaSuccess) return L.e;
  return cudaGetLastError();
}

cudaError_t launch_iteration(const Args& a, const Plan& p, cudaStream_t s, cudaEvent_t (*ev)[2]) {
  return launch_step(a, p, s, VAR_RUNTIME, Handles(), ev);
}

cudaError_t launch_step_var(const Args& a, const Plan& p, cudaStream_t s, int var, cudaEvent_t (*ev)[2]) {
  return launch_step(a, p, s, var, Handles(), ev);
}

cudaError_t launch_step_fused(const Args& a, const Plan& p, cudaStream_t s, int var, bool k1, int fuse_next,
                              cudaEvent_t (*ev)[2]) {
  StepShape sh;
  sh.k1 = k1;
  sh.fuse_next = fuse_next;
  return launch_step(a, p, s, var, Handles(), ev, false, sh);
}

// kernels before a Q pass of a plain step: the factor pre-pass, the tiled factor kernels and
// the two contractions of a QAP product
static int pre_kernels(const Args& a) {
  return (pre_has_work(a, 1, 0) ? 1 : 0) + 3 * tiled_terms(a) + (a.Q.qap_d ? 2 : 0);
}

int kernels_per_step(const Args& a) {
  const bool HQ = a.Q.present(), HA = a.m > 0;
  int k = 1;
  if (HQ) k += 1 + pre_kernels(a);
  if (HA) k += 2 + (HQ ? 1 + pre_kernels(a) : 0);
  if (!HQ && !HA) k += 1;
  return k;
}
int kernels_per_restart(const Args& a) {
  return 1 + ((a.Q.present() && a.m > 0 && a.Q.has_pre())
                  ? (pre_has_work(a, 2, 0) ? 1 : 0) + 2 * tiled_terms(a) + (a.Q.qap_d ? 3 : 0)
                  : 0);
}
int kernels_per_iteration(const Args& a) { return kernels_per_step(a) + kernels_per_restart(a); }

// ------------------------------------------------------------------------------------ dispatch
__global__ void k_dispatch(Args a, Handles hd) {
  if (threadIdx.x == 0 && hd.has_next) cudaGraphSetConditional(hd.sw_next, switch_value(*a.C, hd));
}

static cudaError_t add_cond(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                            unsigned size, cudaGraph_t* bodies) {
  cudaStreamCaptureStatus st;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> dv(deps, deps + nd);
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = size;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, dv.data(), nullptr, dv.size(), &np);
  if (e != cudaSuccess) return e;
  for (unsigned b = 0; b < size; b++) bodies[b] = np.conditional.phGraph_out[b];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// Builds the conditional graph of `steps` inner steps on stream s (side stream s2 captures the
// bodies).  Returns the captured graph in *out.
cudaError_t build_conditional_graph(const Args& a, const Plan& p, cudaStream_t s, cudaStream_t s2, int steps,
                                    cudaGraph_t* out) {
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
  std::vector<cudaGraphConditionalHandle> sw(steps), rs(steps);
  for (int i = 0; i < steps && e == cudaSuccess; i++) {
    e = cudaGraphConditionalHandleCreate(&sw[i], g, 3u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&rs[i], g, 0u, cudaGraphCondAssignDefault);
  }
  if (e == cudaSuccess) {
    Handles h0;
    h0.sw_next = sw[0];
    h0.has_next = 1;
    k_dispatch<<<1, 32, 0, s>>>(a, h0);
    e = cudaGetLastError();
  }
  for (int i = 0; i < steps && e == cudaSuccess; i++) {
    cudaGraph_t bodies[4];
    e = add_cond(s, sw[i], cudaGraphCondTypeSwitch, 4, bodies);
    for (int v = 0; v < 3 && e == cudaSuccess; v++) {
      e = cudaStreamBeginCaptureToGraph(s2, bodies[v], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) break;
      Handles hd;
      hd.rs_cur = rs[i];
      hd.has_rs = 1;
      if (i + 1 < steps) {
        hd.sw_next = sw[i + 1];
        hd.has_next = 1;
      }
      cudaError_t le = launch_step(a, p, s2, v, hd, nullptr);
      cudaGraph_t tmp;
      e = cudaStreamEndCapture(s2, &tmp);
      if (le != cudaSuccess) e = le;
    }
    // body 3 stays empty: nothing to do once the solve is finished
    if (e != cudaSuccess) break;
    cudaGraph_t rb[1];
    e = add_cond(s, rs[i], cudaGraphCondTypeIf, 1, rb);
    if (e != cudaSuccess) break;
    e = cudaStreamBeginCaptureToGraph(s2, rb[0], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) break;
    cudaError_t le = launch_restart(a, p, s2, nullptr);
    cudaGraph_t tmp;
    e = cudaStreamEndCapture(s2, &tmp);
    if (le != cudaSuccess) e = le;
  }
  cudaGraph_t gout = nullptr;
  cudaError_t ee = cudaStreamEndCapture(s, &gout);
  if (e == cudaSuccess) e = ee;
  if (e != cudaSuccess) {
    if (gout) cudaGraphDestroy(gout);
    cudaGetLastError();
    return e;
  }
  *out = gout;
  return cudaSuccess;
}

// Graph of L inner steps with the step variants fixed by position (L a common multiple of
// restart_every and check_every, launched only at iteration counts that are multiples of L):
// the R~ test at multiples of restart_every, the stopping test at multiples of check_every.
// The only data-dependent choice, whether a restart happened at the step before (then the
// restart pass of Algorithm 5 runs and the next step records R~_{r,0}), is one SWITCH node
// after every R~ test; the dynamic graph above spends a SWITCH and an IF node on every step.
cudaError_t build_fixed_graph(const Args& a, const Plan& p, cudaStream_t s, cudaStream_t s2, int L, int re, int ce,
                              cudaGraph_t* out, int* kernels) {
  int nk = 0;   // kernels of one launch in which no restart happens (body 0 of every SWITCH)
  auto sR = [&](int q) { return q % re == 0; };
  auto sT = [&](int q) { return q % ce == 0; };
  auto is_sw = [&](int q) { return sR(q == 1 ? L : q - 1); };
  auto var0 = [&](int q) { return sT(q) ? (int)VAR_T : sR(q) ? (int)VAR_R : (int)VAR_PLAIN; };
  auto varR = [&](int q) { return sT(q) ? (int)VAR_T : (int)VAR_R; };
  // With p.fuse, a step followed by a step without a SWITCH node (no restart can happen in
  // between) runs that step's k_zx at its end: a plain step in K_Q2H, another variant as a
  // separate launch; the step after it then starts with K2.  The step after a SWITCH node (or
  // the first of the graph) runs its own k_zx in every body.
  auto next_sw = [&](int q) { return q == L ? true : is_sw(q + 1); };
  auto shape = [&](int q, int v) {
    StepShape sh;
    sh.k1 = !(p.fuse && q > 1 && !is_sw(q));
    if (p.fuse && !next_sw(q)) {
      if (v == VAR_PLAIN) sh.fuse_next = var0(q + 1);
      else sh.k1_after = var0(q + 1);
    }
    return sh;
  };
  cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed);
  if (e != cudaSuccess) return e;
  cudaStreamCaptureStatus st;
  cudaGraph_t g = nullptr;
  e = cudaStreamGetCaptureInfo(s, &st, nullptr, &g, nullptr, nullptr, nullptr);
  std::vector<cudaGraphConditionalHandle> sw(L + 1);
  for (int q = 1; q <= L && e == cudaSuccess; q++)
    if (is_sw(q)) e = cudaGraphConditionalHandleCreate(&sw[q], g, 3u, cudaGraphCondAssignDefault);
  if (e == cudaSuccess) {
    Handles h0;
    h0.fixed = 1;
    h0.sw_next = sw[1];
    h0.has_next = is_sw(1) ? 1 : 0;
    k_dispatch<<<1, 32, 0, s>>>(a, h0);
    e = cudaGetLastError();
  }
  for (int q = 1; q <= L && e == cudaSuccess; q++) {
    Handles hd;
    hd.fixed = 1;
    if (q < L && is_sw(q + 1)) {
      hd.sw_next = sw[q + 1];
      hd.has_next = 1;
    }
    if (!is_sw(q)) {
      // directly after the previous step's last kernel unless that step sat in a SWITCH body
      StepShape sh = shape(q, var0(q));
      sh.kernels = &nk;
      e = launch_step(a, p, s, var0(q), hd, nullptr, q > 1 && !is_sw(q - 1), sh);
      continue;
    }
    cudaGraph_t bodies[4];
    e = add_cond(s, sw[q], cudaGraphCondTypeSwitch, 4, bodies);
    for (int v = 0; v < 3 && e == cudaSuccess; v++) {
      e = cudaStreamBeginCaptureToGraph(s2, bodies[v], nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
      if (e != cudaSuccess) break;
      cudaError_t le = v == 2 ? launch_restart(a, p, s2, nullptr) : cudaSuccess;
      const int vv = v == 0 ? var0(q) : varR(q);
      StepShape sh = shape(q, vv);
      if (v == 0) sh.kernels = &nk;
      if (le == cudaSuccess) le = launch_step(a, p, s2, vv, hd, nullptr, false, sh);
      cudaGraph_t tmp;
      e = cudaStreamEndCapture(s2, &tmp);
      if (le != cudaSuccess) e = le;
    }
    // body 3 stays empty: the solve is finished
  }
  cudaGraph_t gout = nullptr;
  cudaError_t ee = cudaStreamEndCapture(s, &gout);
  if (e == cudaSuccess) e = ee;
  if (e != cudaSuccess) {
    if (gout) cudaGraphDestroy(gout);
    cudaGetLastError();
    return e;
  }
  *out = gout;
  if (kernels) *kernels = nk + 1;   // + the dispatch kernel
  return cudaSuccess;
}

// ------------------------------------------------------------------------------------ apply / power
cudaError_t launch_apply(const Args& a, const Plan& p, int op, cudaStream_t s) {
  const Handles none;
  if (op == 0) {
    rowk(K_APPLY_A, 0, p.gA)<<<p.gridM, kThreads, 0, s>>>(a, none);
  } else if (op == 1) {
    rowk(K_APPLY_AT, 0, p.gAT)<<<p.gridN, kThreads, 0, s>>>(a, none);
  } else {
    if (pre_has_work(a, 3, 0)) prek(p.gPre, 0)<<<p.gridPre, kThreads, 0, s>>>(a, 3);
    {
      cudaError_t qe = tiled_terms(a) ? launch_tiled(a, p, 3, 0, s, nullptr) : cudaSuccess;
      if (qe == cudaSuccess) qe = launch_qap(a, p, 3, 0, s);
      if (qe != cudaSuccess) return qe;
    }
    rowk(K_APPLY_Q, 0, p.gQ)<<<p.gridN, kThreads, 0, s>>>(a, none);
  }
  return cudaGetLastError();
}

__global__ void k_pw_start(Args a, int64_t dim) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < dim; i += stride) {
    // 0.5 + (hash(i) mod 2^32) / 2^32, a fixed pseudo-random start vector (the w that the
    // first iteration reads, from pv)
    const uint32_t h = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
    a.V.pv[i] = 0.5 + (double)h / 4294967296.0;
  }
}

// which 0: lambda_1(A A^*) on R^m; 1: lambda_1(Q) on R^n
cudaError_t launch_power_init(const Args& a, const Plan& p, int which, cudaStream_t s) {
  const int64_t dim = which == 0 ? a.m : a.n;
  k_pw_start<<<p.gridE, kThreads, 0, s>>>(a, dim);
  return cudaGetLastError();
}

int kernels_per_power_iter(const Args& a, int which) {
  if (which == 0) return 2;
  return 1 + (pre_has_work(a, 4, 0) ? 1 : 0) + 3 * tiled_terms(a) + (a.Q.qap_d ? 2 : 0);
}

// One power iteration, Sec. 4.1: w_{i+1} = M v_i with v_i = w_i / ||w_i||, M = Q or A A^*.  The
// normalisation is folded into the product (M v = pw_scale M w, the scale of the previous w set
// by the last block of the previous product), so w_i and w_{i+1} alternate between pv and pw:
// iteration i reads V.pv and writes V.pw of an Args whose two are swapped when i is odd.
cudaError_t launch_power_iter(const Args& a0, const Plan& p, int which, int i, cudaStream_t s) {
  Args a = a0;
  if (i & 1) std::swap(a.V.pv, a.V.pw);
  const Handles none;
  if (which == 0) {
    rowk(K_APPLY_AT_P, 0, p.gAT)<<<p.gridN, kThreads, 0, s>>>(a, none);
    rowk(K_POWER_A, 0, p.gA)<<<p.gridM, kThreads, 0, s>>>(a, none);
  } else {
    if (pre_has_work(a, 4, 0)) prek(p.gPre, 0)<<<p.gridPre, kThreads, 0, s>>>(a, 4);
    {
      cudaError_t qe = tiled_terms(a) ? launch_tiled(a, p, 4, 0, s, nullptr) : cudaSuccess;
      if (qe == cudaSuccess) qe = launch_qap(a, p, 4, 0, s);
      if (qe != cudaSuccess) return qe;
    }
    rowk(K_POWER_Q, 0, p.gQ)<<<p.gridN, kThreads, 0, s>>>(a, none);
  }
  return cudaGetLastError();
}

// zbar = (xbar - r_z)/sigma from the stored iterate (used by hprqp_get)
__global__ void k_zbar(Args a) {
  const Ctrl* C = a.C;
  const Vec& V = a.V;
  const bool HQ = a.Q.present(), HA = a.m > 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < a.n; j += stride) {
    double g = -V.c[j];
    if (HQ) g -= V.Qw[j];
    if (HA) g += V.ATy[j];
    const double rz = fma(C->sigma, g, V.x[j]);
    V.zb[j] = (V.xb[j] - rz) * C->inv_sigma;
  }
}

cudaError_t launch_zbar(const Args& a, const Plan& p, cudaStream_t s) {
  k_zbar<<<p.gridE, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

// plain CSR SpMV used by the schedule autotuner
template <int G>
__global__ void __launch_bounds__(kThreads) k_spmv_probe(Csr M, const double* x, double* y) {
  __shared__ double rs0[kChunk];
  const int64_t nchunks = (M.rows + kChunk - 1) / kChunk;
  for (int64_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const int64_t row0 = ch * kChunk;
    csr_chunk<G, 1>(M, row0, x, nullptr, rs0, nullptr, false);
    __syncthreads();
    const int64_t j = row0 + threadIdx.x;
    if (j < M.rows) y[j] = rs0[threadIdx.x];
    __syncthreads();
  }
}

// the factor pre-pass t = B_f ain (which = 3) at G lanes per row, for the schedule autotuner
cudaError_t launch_pre_probe(const Args& a, int G, int grid, cudaStream_t s) {
  prek(G, 0)<<<grid, kThreads, 0, s>>>(a, 3);
  return cudaGetLastError();
}

cudaError_t launch_spmv_probe(const Csr& M, int G, int grid, const double* x, double* y, cudaStream_t s) {
  switch (G) {
    case -1: k_spmv_probe<-1><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 0: k_spmv_probe<0><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 1: k_spmv_probe<1><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 2: k_spmv_probe<2><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 4: k_spmv_probe<4><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 8: k_spmv_probe<8><<<grid, kThreads, 0, s>>>(M, x, y); break;
    case 16: k_spmv_probe<16><<<grid, kThreads, 0, s>>>(M, x, y); break;
    default: k_spmv_probe<32><<<grid, kThreads, 0, s>>>(M, x, y); break;
  }
  return cudaGetLastError();
}

}  // namespace hprqp
