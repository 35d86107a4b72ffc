// C ABI of the single-instance HPR-QP solver (include/hprqp.h).
//
// Host responsibilities: validate and copy the problem (host or device inputs), have the
// device build the stored transposes A^T and B_f^T (each transposed row in increasing original
// row order) and the SELL and tiled copies (sell_build.cu), pick the SpMV schedule, run the
// power method of Sec. 4.1, and drive Algorithm 4 through CUDA graphs (solver.cu) whose kernels
// stop themselves once the device-side controller has set the done flag.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <functional>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hprqp.h"
#include "../../include/hprqp_learn.h"
#include "sell_build.cuh"
#include "solver.cuh"

using namespace hprqp;

struct hprqp_handle {
  int dev = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  hprqp_params prm;
  int64_t n = 0, m = 0;
  int phi = 0;
  double lambda = 0.0;
  std::vector<std::pair<void*, size_t>> allocs;
  Args args;
  Plan plan;
  Ctrl* dctrl = nullptr;
  Ctrl* hctrl = nullptr;      // pinned mirror
  int* hflags = nullptr;      // pinned done flags
  double nb2 = 0, nc2 = 0, b_inf = 0, c_inf = 0;
  std::vector<double> ws_x, ws_y;
  double ws_sigma = 0.0;
  cudaGraphExec_t g_iter = nullptr;
  cudaGraphExec_t g_fixed = nullptr;   // fixed-schedule graph of fixed_L steps (conditional mode)
  int fixed_L = 0;
  int fixed_kernels = 0;          // kernels of one fixed-graph launch without restarts
  int64_t fixed_steps = 0;        // inner steps run through the fixed graph in this solve
  bool fixed_tried = false;
  cudaGraphExec_t g_pw[2] = {nullptr, nullptr};
  int pw_chunk = 16;
  // the power method on A A^* runs beside the one on Q (both needed: m > 0 and Q present): its
  // own controller copy, partials, counters and vectors, on its own stream
  bool pw_pair = false;
  Args pwA_args;
  Ctrl* dctrl2 = nullptr;
  Ctrl* hctrl2 = nullptr;     // pinned mirror
  cudaStream_t pstream = nullptr;
  cudaEvent_t pfork = nullptr, pjoin = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  std::string err;
  hprqp_kkt kkt;
  int last_status = -1;
  bool solved = false;
  int64_t launches = 0;
  // device memory of the handle by path: the allocator hooks, or cudaMalloc
  int64_t hook_count = 0, hook_bytes = 0, rt_count = 0, rt_bytes = 0;
  double last_lamA = 0, last_lamQ = 0, last_sigma0 = 1;
  cudaStream_t side = nullptr;   // captures the bodies of the conditional nodes
  bool conditional = false;      // the iteration graph selects step variants on the device
  // preconditioning (Sec. 4.1): x = D xs, y = E ys; host copies of d, e and scratch for the
  // unscaled outputs of hprqp_get
  bool scaled = false;
  std::vector<double> hd, he;
  double *ux = nullptr, *uy = nullptr, *uz = nullptr, *uw = nullptr;
  // primal HPR methods (Appendix A): state allocated at their first solve
  bool primal_ready = false;
  double *px = nullptr, *ps = nullptr, *py = nullptr, *pv = nullptr, *pt = nullptr;
  double *px0 = nullptr, *ps0 = nullptr, *py0 = nullptr, *pv0 = nullptr, *pt0 = nullptr;
  double *pxb = nullptr, *psb = nullptr, *pyb = nullptr, *pvb = nullptr, *ptb = nullptr, *pzb = nullptr;
  double *pAx = nullptr, *pQv = nullptr, *pw = nullptr, *pATw = nullptr, *pAxb = nullptr, *pQxb = nullptr,
         *pATyb = nullptr, *ppn = nullptr, *ppm = nullptr, *pout = nullptr;
};

static thread_local std::string g_create_err;

// NVTX range for profilers (setup, power method, iteration, output); free when none attaches
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// ------------------------------------------------------------------------------------ helpers
static hprqp_status fail(hprqp_handle* h, hprqp_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (h) h->err = buf;
  else g_create_err = buf;
  return st;
}

#define CU(h, call)                                                                          \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      cudaGetLastError();                                                                    \
      return fail(h, e_ == cudaErrorMemoryAllocation ? HPRQP_OOM : HPRQP_CUDA_ERROR, "%s: %s (%s:%d)", #call, \
                  cudaGetErrorString(e_), __FILE__, __LINE__);                               \
    }                                                                                        \
  } while (0)

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class T>
static hprqp_status fetch(hprqp_handle* h, std::vector<T>& out, const T* p, size_t count) {
  out.resize(count);
  if (count == 0) return HPRQP_OK;
  if (!p) return fail(h, HPRQP_INVALID_ARG, "null input pointer for %zu elements", count);
  if (is_device_ptr(p)) {
    CU(h, cudaMemcpy(out.data(), p, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(out.data(), p, count * sizeof(T));
  }
  return HPRQP_OK;
}

static hprqp_status dalloc(hprqp_handle* h, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  bytes = (bytes + 255) / 256 * 256;
  if (h->prm.alloc) {
    *p = h->prm.alloc(bytes, h->prm.alloc_ctx, h->stream);
    if (!*p) return fail(h, HPRQP_OOM, "allocator hook returned NULL for %zu bytes", bytes);
    h->hook_count++;
    h->hook_bytes += (int64_t)bytes;
  } else {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(h, HPRQP_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
    h->rt_count++;
    h->rt_bytes += (int64_t)bytes;
  }
  h->allocs.push_back({*p, bytes});
  return HPRQP_OK;
}

template <class T>
static hprqp_status upload(hprqp_handle* h, T** dst, const std::vector<T>& src, size_t min_count = 1) {
  void* p = nullptr;
  size_t cnt = std::max(src.size(), min_count);
  hprqp_status st = dalloc(h, &p, cnt * sizeof(T));
  if (st) return st;
  if (!src.empty()) CU(h, cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, h->stream));
  if (cnt > src.size()) CU(h, cudaMemsetAsync((T*)p + src.size(), 0, (cnt - src.size()) * sizeof(T), h->stream));
  *dst = (T*)p;
  return HPRQP_OK;
}

static hprqp_status zeros(hprqp_handle* h, double** dst, size_t count) {
  void* p = nullptr;
  hprqp_status st = dalloc(h, &p, std::max<size_t>(count, 1) * sizeof(double));
  if (st) return st;
  CU(h, cudaMemsetAsync(p, 0, std::max<size_t>(count, 1) * sizeof(double), h->stream));
  *dst = (double*)p;
  return HPRQP_OK;
}

struct HostCsr {
  int64_t rows = 0, cols = 0;
  std::vector<int> rp, ci;
  std::vector<double> v;
};

static hprqp_status check_csr(hprqp_handle* h, const HostCsr& M, const char* name) {
  if ((int64_t)M.rp.size() != M.rows + 1) return fail(h, HPRQP_INVALID_ARG, "%s: row pointer size", name);
  if (M.rp[0] != 0) return fail(h, HPRQP_INVALID_ARG, "%s: row pointers must start at 0", name);
  for (int64_t i = 0; i < M.rows; i++)
    if (M.rp[i + 1] < M.rp[i]) return fail(h, HPRQP_INVALID_ARG, "%s: row pointers decrease at row %lld", name, (long long)i);
  const int64_t nnz = M.rp[M.rows];
  if ((int64_t)M.ci.size() != nnz || (int64_t)M.v.size() != nnz) return fail(h, HPRQP_INVALID_ARG, "%s: nnz mismatch", name);
  for (int64_t k = 0; k < nnz; k++) {
    if (M.ci[k] < 0 || M.ci[k] >= M.cols)
      return fail(h, HPRQP_INVALID_ARG, "%s: column index %d out of range at entry %lld", name, M.ci[k], (long long)k);
    if (!std::isfinite(M.v[k])) return fail(h, HPRQP_INVALID_ARG, "%s: non-finite value at entry %lld", name, (long long)k);
  }
  return HPRQP_OK;
}

// deterministic transpose: entries of each transposed row in increasing original-row order
static HostCsr transpose(const HostCsr& M) {
  HostCsr T;
  T.rows = M.cols;
  T.cols = M.rows;
  const int64_t nnz = M.rp[M.rows];
  T.rp.assign(T.rows + 1, 0);
  for (int64_t k = 0; k < nnz; k++) T.rp[M.ci[k] + 1]++;
  for (int64_t i = 0; i < T.rows; i++) T.rp[i + 1] += T.rp[i];
  std::vector<int> pos(T.rp.begin(), T.rp.end() - 1);
  T.ci.resize(nnz);
  T.v.resize(nnz);
  for (int64_t r = 0; r < M.rows; r++)
    for (int k = M.rp[r]; k < M.rp[r + 1]; k++) {
      int c = M.ci[k];
      T.ci[pos[c]] = (int)r;
      T.v[pos[c]] = M.v[k];
      pos[c]++;
    }
  return T;
}

// SELL-32-512 copy of the device CSR matrix d tile by tile over its columns (tile k: columns
// [k W, (k+1) W), W = kTileW, at most kMaxTilesDevice tiles), built on the device: per tile,
// rows in windows of 512 sorted by their entry count in the tile (ties by row), slices of 32
// rows padded with zero values to the slice's longest row, a row's entries in their order
// inside the row, column indices relative to the tile.
static hprqp_status build_sell_dev(hprqp_handle* h, SellTiles& S, const Csr& d) {
  static_assert(kTileW <= 65536, "tile-local columns must fit 16 bits");
  const int64_t rows = d.rows, nsl = (rows + 31) / 32;
  const int nt = (int)std::max<int64_t>(1, (d.cols + kTileW - 1) / kTileW);
  if (nt > kMaxTilesDevice || rows == 0) return fail(h, HPRQP_INVALID_ARG, "tiled factor copy: shape");
  hprqp_status st;
  void *len, *perm, *slot, *width, *off, *total;
  if ((st = dalloc(h, &len, (size_t)nt * rows * sizeof(int))) ||
      (st = dalloc(h, &perm, (size_t)nt * nsl * 32 * sizeof(int))) ||
      (st = dalloc(h, &slot, (size_t)nt * rows * sizeof(int))) ||
      (st = dalloc(h, &width, (size_t)nt * nsl * sizeof(int))) ||
      (st = dalloc(h, &off, (size_t)nt * (nsl + 1) * sizeof(int))) || (st = dalloc(h, &total, sizeof(long long))))
    return st;
  CU(h, tile_layout(d, kTileW, nt, (int*)len, (int*)perm, (int*)slot, (int*)width, (int*)off, (long long*)total,
                    h->stream));
  long long tot = 0;
  CU(h, cudaMemcpyAsync(&tot, total, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (tot < 0 || tot >= ((long long)1 << 31)) return fail(h, HPRQP_INVALID_ARG, "tiled factor copy: too many entries");
  void *col, *val;
  const size_t cnt = (size_t)std::max<long long>(tot, 1);
  if ((st = dalloc(h, &col, cnt * sizeof(unsigned short))) || (st = dalloc(h, &val, cnt * sizeof(double)))) return st;
  CU(h, cudaMemsetAsync(col, 0, cnt * sizeof(unsigned short), h->stream));
  CU(h, cudaMemsetAsync(val, 0, cnt * sizeof(double), h->stream));
  CU(h, tile_fill(d, kTileW, nt, (const int*)slot, (const int*)off, (unsigned short*)col, (double*)val, h->stream));
  S.rows = rows;
  S.ntile = nt;
  S.nsl = nsl;
  S.off = (const int*)off;
  S.perm = (const int*)perm;
  S.col = (const unsigned short*)col;
  S.val = (const double*)val;
  return HPRQP_OK;
}

// Tiled copies of a factor term B (p x n) for the shared-memory products of tiled.cu: B tiled
// over its columns (the entries of x), B^T over its columns (the entries of t = B x); from
// the device copies dB, dBT of B and B^T.
static hprqp_status build_tiled(hprqp_handle* h, TiledFac& T, const Csr& dB, const Csr& dBT, int sms) {
  hprqp_status st;
  if ((st = build_sell_dev(h, T.b, dB)) || (st = build_sell_dev(h, T.bt, dBT))) return st;
  T.p = dB.rows;
  const int64_t nwin = (T.b.nsl + kSellWin / kSellC - 1) / (kSellWin / kSellC);
  // one wave of (tile, window range) blocks at one block per SM
  T.nrange = (int)std::max<int64_t>(1, std::min<int64_t>(sms / T.b.ntile, nwin));
  return zeros(h, &T.part, (size_t)T.b.ntile * (size_t)dB.rows);
}

// SELL-32 copy of a device CSR matrix for the row passes, built on the device (sorting
// windows = the 256-row chunks of the row kernels, so a chunk's slices hold exactly its rows).
static hprqp_status build_sell_rows(hprqp_handle* h, Csr& d) {
  const int64_t nsl = (d.rows + 31) / 32;
  hprqp_status st;
  void *perm, *width, *off, *total;
  if ((st = dalloc(h, &perm, (size_t)nsl * 32 * sizeof(int))) || (st = dalloc(h, &width, (size_t)nsl * sizeof(int))) ||
      (st = dalloc(h, &off, (size_t)(nsl + 1) * sizeof(int))) || (st = dalloc(h, &total, sizeof(long long))))
    return st;
  CU(h, sell_layout(d, (int*)perm, (int*)width, (int*)off, (long long*)total, h->stream));
  long long tot = 0;
  CU(h, cudaMemcpyAsync(&tot, total, sizeof(long long), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (tot < 0 || tot >= ((long long)1 << 31)) return fail(h, HPRQP_INVALID_ARG, "SELL copy: too many entries");
  void *sci, *sv;
  if ((st = dalloc(h, &sci, (size_t)std::max<long long>(tot, 1) * sizeof(int))) ||
      (st = dalloc(h, &sv, (size_t)std::max<long long>(tot, 1) * sizeof(double))))
    return st;
  CU(h, cudaMemsetAsync(sci, 0, (size_t)std::max<long long>(tot, 1) * sizeof(int), h->stream));
  CU(h, cudaMemsetAsync(sv, 0, (size_t)std::max<long long>(tot, 1) * sizeof(double), h->stream));
  CU(h, sell_fill(d, (const int*)perm, (const int*)off, (int*)sci, (double*)sv, h->stream));
  d.soff = (const int*)off;
  d.sperm = (const int*)perm;
  d.sci = (const int*)sci;
  d.sv = (const double*)sv;
  return HPRQP_OK;
}

static hprqp_status upload_csr(hprqp_handle* h, Csr& d, const HostCsr& M) {
  d.rows = M.rows;
  d.cols = M.cols;
  d.nnz = M.rp.empty() ? 0 : M.rp[M.rows];
  int *rp, *ci;
  double* v;
  hprqp_status st;
  if ((st = upload(h, &rp, M.rp))) return st;
  if ((st = upload(h, &ci, M.ci))) return st;
  if ((st = upload(h, &v, M.v))) return st;
  d.rp = rp;
  d.ci = ci;
  d.v = v;
  return HPRQP_OK;
}

// Stored transpose of a matrix already on the device (d), built on the device in the order of
// the host counting sort; the host transpose of M when a transposed row would hold more than
// 2048 entries (the device sorts each row by insertion).
static hprqp_status upload_transpose(hprqp_handle* h, Csr& t, const Csr& d, const HostCsr& M) {
  hprqp_status st;
  void *rp, *mx;
  if ((st = dalloc(h, &rp, (size_t)(d.cols + 1) * sizeof(int))) || (st = dalloc(h, &mx, sizeof(int)))) return st;
  CU(h, transpose_layout(d, (int*)rp, (int*)mx, h->stream));
  int maxlen = 0;
  CU(h, cudaMemcpyAsync(&maxlen, mx, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  if (maxlen > 2048) return upload_csr(h, t, transpose(M));
  void *cur, *ci, *v;
  if ((st = dalloc(h, &cur, (size_t)std::max<int64_t>(d.cols, 1) * sizeof(int))) ||
      (st = dalloc(h, &ci, (size_t)std::max<int64_t>(d.nnz, 1) * sizeof(int))) ||
      (st = dalloc(h, &v, (size_t)std::max<int64_t>(d.nnz, 1) * sizeof(double))))
    return st;
  CU(h, transpose_fill(d, (const int*)rp, (int*)cur, (int*)ci, (double*)v, h->stream));
  t.rows = d.cols;
  t.cols = d.rows;
  t.nnz = d.nnz;
  t.rp = (const int*)rp;
  t.ci = (const int*)ci;
  t.v = (const double*)v;
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ defaults
extern "C" void hprqp_default_params(hprqp_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->stream = nullptr;
  p->check_every = 100;
  p->restart_every = 10;
  p->alpha1 = 0.2;
  p->alpha2 = 0.8;
  p->alpha3 = 0.5;
  p->alpha3_tight = 0.2;
  p->ratio_tight = 0.1;
  p->lambda_A = 0.0;
  p->lambda_Q = 0.0;
  p->sigma0 = 0.0;
  p->power_max_iter = 5000;
  p->power_tol = 1e-6;
  p->power_safety = 1.01;
  p->time_limit = 0.0;
  p->iters_per_launch = 64;
  p->autotune = 1;
  p->scaling = 1;
  p->method = 0;
  p->pdl = 1;
  p->fixed_schedule = 1;
  p->tiled_factor = 1;
  p->fused_steps = 1;
  p->factor_inline = 1;
}

extern "C" const char* hprqp_last_error(const hprqp_handle* h) {
  return h ? h->err.c_str() : g_create_err.c_str();
}

static void release(hprqp_handle* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  if (h->g_iter) cudaGraphExecDestroy(h->g_iter);
  if (h->g_fixed) cudaGraphExecDestroy(h->g_fixed);
  for (auto& g : h->g_pw)
    if (g) cudaGraphExecDestroy(g);
  for (auto& e : h->ev)
    if (e) cudaEventDestroy(e);
  if (h->pstream) {
    cudaStreamSynchronize(h->pstream);
    cudaStreamDestroy(h->pstream);
  }
  if (h->pfork) cudaEventDestroy(h->pfork);
  if (h->pjoin) cudaEventDestroy(h->pjoin);
  for (auto& a : h->allocs) {
    if (h->prm.free) h->prm.free(a.first, a.second, h->prm.alloc_ctx, h->stream);
    else cudaFree(a.first);
  }
  if (h->hctrl) cudaFreeHost(h->hctrl);
  if (h->hctrl2) cudaFreeHost(h->hctrl2);
  if (h->hflags) cudaFreeHost(h->hflags);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  cudaGetLastError();
  delete h;
}

extern "C" void hprqp_destroy(hprqp_handle* h) { release(h); }

extern "C" hprqp_status hprqp_memory_stats(const hprqp_handle* h, int64_t* out) {
  if (!h || !out) return HPRQP_INVALID_ARG;
  out[0] = h->hook_count;
  out[1] = h->hook_bytes;
  out[2] = h->rt_count;
  out[3] = h->rt_bytes;
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ autotune
static int tune_G(hprqp_handle* h, const Csr& M, int grid, double* x, double* y, int fallback) {
  if (M.rows == 0 || M.nnz == 0) return fallback;
  if (h->prm.autotune == 2) return 0;
  if (h->prm.autotune == 3) return M.soff ? -1 : 1;
  if (!h->prm.autotune) {
    double avg = (double)M.nnz / (double)M.rows;
    return avg < 6 ? 1 : avg < 12 ? 2 : avg < 24 ? 4 : avg < 64 ? 8 : 32;
  }
  // lanes per row (1-32), 0: the staged form that streams each chunk's entries as a block,
  // -1: the SELL copy (A and A^T)
  const int cand[8] = {-1, 0, 1, 2, 4, 8, 16, 32};
  float best = 1e30f;
  int bestG = fallback;
  for (int G : cand) {
    if (G == -1 && !M.soff) continue;
    launch_spmv_probe(M, G, grid, x, y, h->stream);
    float tot = 0;
    for (int r = 0; r < 3; r++) {
      cudaEventRecord(h->ev[0], h->stream);
      launch_spmv_probe(M, G, grid, x, y, h->stream);
      cudaEventRecord(h->ev[1], h->stream);
      cudaEventSynchronize(h->ev[1]);
      float ms = 0;
      cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]);
      tot += ms;
    }
    if (cudaGetLastError() != cudaSuccess) continue;
    // the probe is a bare SpMV; inside the row kernels the SELL form also frees the
    // epilogue's loads from uncoalesced index traffic, so it wins ties within 10 %
    if (G == -1) tot *= 0.9f;
    if (tot < best) {
      best = tot;
      bestG = G;
    }
  }
  return bestG;
}

// ------------------------------------------------------------------------------------ create
// Checks c (finite) and the row bounds (l <= u, no NaN) and records the norms that the
// stopping test (Sec. 4.1: b = max(|l|, |u|) with infinite entries as 0) and the sigma0
// rule use.
static hprqp_status data_norms(hprqp_handle* h, const std::vector<double>& hc, const std::vector<double>& hl,
                               const std::vector<double>& hu) {
  for (size_t j = 0; j < hc.size(); j++)
    if (!std::isfinite(hc[j])) return fail(h, HPRQP_INVALID_ARG, "c[%lld] is not finite", (long long)j);
  double nb2 = 0, bi = 0;
  for (size_t i = 0; i < hl.size(); i++) {
    // K = {y real : l <= y <= u} (Sec. 1): l = +inf or u = -inf leaves it empty
    if (std::isnan(hl[i]) || std::isnan(hu[i]) || hl[i] > hu[i] || hl[i] == INFINITY || hu[i] == -INFINITY)
      return fail(h, HPRQP_INVALID_ARG, "row bound %lld: need l <= u, l < +inf, u > -inf, no NaN", (long long)i);
    double bl = std::isfinite(hl[i]) ? std::fabs(hl[i]) : 0.0;
    double bu = std::isfinite(hu[i]) ? std::fabs(hu[i]) : 0.0;
    double b = std::max(bl, bu);
    nb2 += b * b;
    bi = std::max(bi, b);
  }
  double nc2 = 0, ci = 0;
  for (double v : hc) {
    nc2 += v * v;
    ci = std::max(ci, std::fabs(v));
  }
  h->nb2 = nb2;
  h->nc2 = nc2;
  h->b_inf = bi;
  h->c_inf = ci;
  return HPRQP_OK;
}

// Scratch of the QAP term's split contractions (qap.cu): partial tiles and per-tile counters
static hprqp_status qap_scratch(hprqp_handle* h, QDev& QD) {
  int dev = 0, sms = 0;
  CU(h, cudaGetDevice(&dev));
  CU(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t d = QD.qap_d, tiles_i = (d + 31) / 32;
  QD.qap_splits = qap_splits(d, sms);
  void* p = nullptr;
  hprqp_status st;
  if ((st = dalloc(h, &p, sizeof(double) * (size_t)QD.qap_splits * d * d))) return st;
  QD.qap_part = (double*)p;
  if ((st = dalloc(h, &p, sizeof(unsigned) * (size_t)(tiles_i * tiles_i)))) return st;
  CU(h, cudaMemsetAsync(p, 0, sizeof(unsigned) * (size_t)(tiles_i * tiles_i), h->stream));
  QD.qap_count = (unsigned*)p;
  return HPRQP_OK;
}

// Sec. 4.1 preconditioning: ten Ruiz passes (infinity norms), then one Pock-Chambolle pass
// with alpha = 1 (1-norms), on the symmetric K = [Q A^T; A 0] scaled as diag(s) K diag(s),
// s = (d, e); every pass divides s_j by the square root of the norm of column j of the
// currently scaled K (norm 0: s_j unchanged).  Q given by its diagonal, merged CSR and bands.
static void precondition(int64_t n, int64_t m, const std::vector<double>& qdiag, const HostCsr& qcsr,
                         const std::vector<int>& dia_off, const std::vector<std::vector<double>>& dia_vals,
                         const HostCsr& A, std::vector<double>& d, std::vector<double>& e) {
  d.assign(n, 1.0);
  e.assign(m, 1.0);
  std::vector<double> cn(n), rn(m);
  for (int pass = 0; pass < 11; pass++) {
    const bool ruiz = pass < 10;
    std::fill(cn.begin(), cn.end(), 0.0);
    std::fill(rn.begin(), rn.end(), 0.0);
    auto put = [ruiz](double& acc, double v) { acc = ruiz ? std::max(acc, std::fabs(v)) : acc + std::fabs(v); };
    if (!qdiag.empty())
      for (int64_t j = 0; j < n; j++) put(cn[j], qdiag[j] * d[j] * d[j]);
    if (qcsr.rows)
      for (int64_t i = 0; i < n; i++)        // symmetric: column i has the norm of row i
        for (int k = qcsr.rp[i]; k < qcsr.rp[i + 1]; k++) put(cn[i], qcsr.v[k] * d[i] * d[qcsr.ci[k]]);
    for (size_t b = 0; b < dia_off.size(); b++) {
      const int64_t o = dia_off[b];
      for (int64_t i = 0; i + o < n; i++) {
        const double v = dia_vals[b][i] * d[i] * d[i + o];
        put(cn[i], v);
        if (o != 0) put(cn[i + o], v);
      }
    }
    for (int64_t i = 0; i < m; i++)
      for (int k = A.rp[i]; k < A.rp[i + 1]; k++) {
        const double v = A.v[k] * e[i] * d[A.ci[k]];
        put(cn[A.ci[k]], v);
        put(rn[i], v);
      }
    for (int64_t j = 0; j < n; j++)
      if (cn[j] > 0.0) d[j] /= std::sqrt(cn[j]);
    for (int64_t i = 0; i < m; i++)
      if (rn[i] > 0.0) e[i] /= std::sqrt(rn[i]);
  }
}

// c_s = D c, [l_s, u_s] = E [l, u] (in place) and the norms of the sigma0 rule on them
static void scale_data(hprqp_handle* h, std::vector<double>& hc, std::vector<double>& hl, std::vector<double>& hu) {
  for (size_t j = 0; j < hc.size(); j++) hc[j] *= h->hd[j];
  for (size_t i = 0; i < hl.size(); i++) {
    hl[i] *= h->he[i];
    hu[i] *= h->he[i];
  }
  double nb2 = 0.0, nc2 = 0.0;
  for (size_t i = 0; i < hl.size(); i++) {
    const double b = std::max(std::isfinite(hl[i]) ? std::fabs(hl[i]) : 0.0, std::isfinite(hu[i]) ? std::fabs(hu[i]) : 0.0);
    nb2 += b * b;
  }
  for (double v : hc) nc2 += v * v;
  h->nb2 = nb2;
  h->nc2 = nc2;
}

// verbose >= 2: wall time of each phase of hprqp_create on stderr (device work synchronised)
struct PhaseClock {
  hprqp_handle* h;
  std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
  void mark(const char* name) {
    if (h->prm.verbose < 2) return;
    cudaStreamSynchronize(h->stream);
    const auto now = std::chrono::steady_clock::now();
    std::fprintf(stderr, "hprqp_create: %-16s %8.2f ms\n", name,
                 std::chrono::duration<double, std::milli>(now - t).count());
    t = now;
  }
};

static hprqp_status create_impl(hprqp_handle* h, int64_t n, int64_t m, const hprqp_qop* Q, const int32_t* A_rowptr,
                                const int32_t* A_colidx, const double* A_vals, const double* c, const double* l,
                                const double* u, const double* L, const double* U, int32_t phi, double lambda) {
  hprqp_status st;
  PhaseClock clk{h};
  if (n <= 0 || m < 0) return fail(h, HPRQP_INVALID_ARG, "need n > 0 and m >= 0 (n=%lld, m=%lld)", (long long)n, (long long)m);
  if (n >= (int64_t)1 << 31 || m >= (int64_t)1 << 31) return fail(h, HPRQP_INVALID_ARG, "n and m must be < 2^31");
  if (phi < 0 || phi > 2) return fail(h, HPRQP_INVALID_ARG, "unknown phi kind %d", phi);
  if (phi != PHI_BOX && !(lambda >= 0.0 && std::isfinite(lambda))) return fail(h, HPRQP_INVALID_ARG, "lambda must be finite and >= 0");
  h->n = n;
  h->m = m;
  h->phi = phi;
  h->lambda = phi == PHI_BOX ? 0.0 : lambda;

  // ---- vectors
  std::vector<double> hc, hl, hu, hL, hU;
  if ((st = fetch(h, hc, c, n))) return st;
  if ((st = fetch(h, hl, l, m))) return st;
  if ((st = fetch(h, hu, u, m))) return st;
  if (L) {
    if ((st = fetch(h, hL, L, n))) return st;
  } else {
    if (phi != PHI_L1) return fail(h, HPRQP_INVALID_ARG, "L is required for box constraints");
    hL.assign(n, -INFINITY);
  }
  if (U) {
    if ((st = fetch(h, hU, U, n))) return st;
  } else {
    if (phi != PHI_L1) return fail(h, HPRQP_INVALID_ARG, "U is required for box constraints");
    hU.assign(n, INFINITY);
  }
  if (phi == PHI_L1) {
    hL.assign(n, -INFINITY);
    hU.assign(n, INFINITY);
  }
  for (int64_t j = 0; j < n; j++) {
    // L in (R u {-inf})^n, U in (R u {+inf})^n (Sec. 1)
    if (std::isnan(hL[j]) || std::isnan(hU[j]) || hL[j] > hU[j] || hL[j] == INFINITY || hU[j] == -INFINITY)
      return fail(h, HPRQP_INVALID_ARG, "box bound %lld: need L <= U, L < +inf, U > -inf, no NaN", (long long)j);
  }
  if ((st = data_norms(h, hc, hl, hu))) return st;

  clk.mark("vectors");
  // ---- A
  HostCsr A;
  A.rows = m;
  A.cols = n;
  if (m > 0) {
    if ((st = fetch(h, A.rp, A_rowptr, m + 1))) return st;
    if (A.rp[0] != 0 || A.rp[m] < 0) return fail(h, HPRQP_INVALID_ARG, "A: bad row pointers");
    int64_t nnz = A.rp[m];
    if ((st = fetch(h, A.ci, A_colidx, nnz))) return st;
    if ((st = fetch(h, A.v, A_vals, nnz))) return st;
    if ((st = check_csr(h, A, "A"))) return st;
  }

  clk.mark("A");
  // ---- Q terms
  std::vector<double> qdiag;
  HostCsr qcsr;
  qcsr.rows = 0;
  std::vector<int> dia_off;
  std::vector<std::vector<double>> dia_vals;
  std::vector<HostCsr> facs;
  std::vector<std::pair<int64_t, std::vector<double>>> dens;
  int64_t qap_d = 0;
  std::vector<double> qap_vals;
  std::vector<HostCsr> csr_terms;
  int nterms = Q ? Q->nterms : 0;
  if (nterms < 0 || (nterms > 0 && !Q->terms)) return fail(h, HPRQP_INVALID_ARG, "bad Q operator");
  for (int t = 0; t < nterms; t++) {
    const hprqp_qterm& q = Q->terms[t];
    if (q.kind == HPRQP_Q_DIAG) {
      std::vector<double> d;
      if ((st = fetch(h, d, q.dense, n))) return st;
      for (double x : d)
        if (!std::isfinite(x)) return fail(h, HPRQP_INVALID_ARG, "Q diag: non-finite value");
      if (qdiag.empty()) qdiag.assign(n, 0.0);
      for (int64_t j = 0; j < n; j++) qdiag[j] += d[j];
    } else if (q.kind == HPRQP_Q_CSR) {
      HostCsr M;
      M.rows = n;
      M.cols = n;
      if ((st = fetch(h, M.rp, q.rowptr, n + 1))) return st;
      if (M.rp[0] != 0 || M.rp[n] < 0) return fail(h, HPRQP_INVALID_ARG, "Q csr: bad row pointers");
      if ((st = fetch(h, M.ci, q.colidx, M.rp[n]))) return st;
      if ((st = fetch(h, M.v, q.vals, M.rp[n]))) return st;
      if ((st = check_csr(h, M, "Q csr"))) return st;
      csr_terms.push_back(std::move(M));
    } else if (q.kind == HPRQP_Q_DIA) {
      if (q.ndiag <= 0 || !q.offsets) return fail(h, HPRQP_INVALID_ARG, "Q dia: need ndiag > 0 and offsets");
      std::vector<int> off;
      std::vector<double> dv;
      if ((st = fetch(h, off, q.offsets, q.ndiag))) return st;
      if ((st = fetch(h, dv, q.diags, (size_t)q.ndiag * n))) return st;
      for (int k = 0; k < q.ndiag; k++) {
        if (off[k] < 0 || off[k] >= n) return fail(h, HPRQP_INVALID_ARG, "Q dia: offset %d out of range", off[k]);
        auto it = std::find(dia_off.begin(), dia_off.end(), off[k]);
        size_t slot;
        if (it == dia_off.end()) {
          if ((int)dia_off.size() >= kMaxDia) return fail(h, HPRQP_INVALID_ARG, "Q dia: at most %d distinct offsets", kMaxDia);
          dia_off.push_back(off[k]);
          dia_vals.emplace_back(n, 0.0);
          slot = dia_off.size() - 1;
        } else {
          slot = it - dia_off.begin();
        }
        for (int64_t i = 0; i + off[k] < n; i++) {
          double x = dv[(size_t)k * n + i];
          if (!std::isfinite(x)) return fail(h, HPRQP_INVALID_ARG, "Q dia: non-finite value");
          dia_vals[slot][i] += x;
        }
      }
    } else if (q.kind == HPRQP_Q_FACTOR) {
      if (q.p <= 0 || q.p >= ((int64_t)1 << 31)) return fail(h, HPRQP_INVALID_ARG, "Q factor: bad p");
      if ((int)facs.size() >= kMaxFac) return fail(h, HPRQP_INVALID_ARG, "at most %d factor terms", kMaxFac);
      HostCsr B;
      B.rows = q.p;
      B.cols = n;
      if ((st = fetch(h, B.rp, q.rowptr, q.p + 1))) return st;
      if (B.rp[0] != 0 || B.rp[q.p] < 0) return fail(h, HPRQP_INVALID_ARG, "Q factor: bad row pointers");
      if ((st = fetch(h, B.ci, q.colidx, B.rp[q.p]))) return st;
      if ((st = fetch(h, B.v, q.vals, B.rp[q.p]))) return st;
      if ((st = check_csr(h, B, "Q factor"))) return st;
      facs.push_back(std::move(B));
    } else if (q.kind == HPRQP_Q_DENSE_FACTOR) {
      if (q.p <= 0) return fail(h, HPRQP_INVALID_ARG, "Q dense factor: bad p");
      if ((int)dens.size() >= kMaxDense) return fail(h, HPRQP_INVALID_ARG, "at most %d dense factor terms", kMaxDense);
      std::vector<double> F;
      if ((st = fetch(h, F, q.dense, (size_t)q.p * n))) return st;
      for (double x : F)
        if (!std::isfinite(x)) return fail(h, HPRQP_INVALID_ARG, "Q dense factor: non-finite value");
      dens.push_back({q.p, std::move(F)});
    } else if (q.kind == HPRQP_Q_QAP) {
      if (qap_d) return fail(h, HPRQP_INVALID_ARG, "at most one QAP term");
      if (q.p <= 0 || q.p * q.p != n) return fail(h, HPRQP_INVALID_ARG, "QAP term: need p = d with n = d^2");
      if (h->prm.launch_mode == 3) return fail(h, HPRQP_INVALID_ARG, "QAP term: not with launch_mode 3");
      if ((st = fetch(h, qap_vals, q.dense, (size_t)4 * q.p * q.p))) return st;
      for (double x : qap_vals)
        if (!std::isfinite(x)) return fail(h, HPRQP_INVALID_ARG, "QAP term: non-finite value");
      qap_d = q.p;
    } else {
      return fail(h, HPRQP_INVALID_ARG, "unknown Q term kind %d", q.kind);
    }
  }
  // several explicit CSR terms: concatenate rows (duplicates are summed by the SpMV)
  if (!csr_terms.empty()) {
    qcsr.rows = n;
    qcsr.cols = n;
    qcsr.rp.assign(n + 1, 0);
    for (int64_t i = 0; i < n; i++) {
      int64_t cnt = 0;
      for (auto& M : csr_terms) cnt += M.rp[i + 1] - M.rp[i];
      qcsr.rp[i + 1] = (int)(qcsr.rp[i] + cnt);
    }
    qcsr.ci.reserve(qcsr.rp[n]);
    qcsr.v.reserve(qcsr.rp[n]);
    for (int64_t i = 0; i < n; i++)
      for (auto& M : csr_terms)
        for (int k = M.rp[i]; k < M.rp[i + 1]; k++) {
          qcsr.ci.push_back(M.ci[k]);
          qcsr.v.push_back(M.v[k]);
        }
  }

  clk.mark("Q terms");
  // ---- preconditioning (Sec. 4.1: only when Q is explicit; the box-only phi keeps the
  // prox a plain clip in the scaled variables).  b_inf, c_inf of the stopping test stay those
  // of the original data; the sigma0 norms become those of the scaled data.
  h->scaled = h->prm.scaling && phi == PHI_BOX && facs.empty() && dens.empty() && qap_d == 0;
  if (h->scaled) {
    precondition(n, m, qdiag, qcsr, dia_off, dia_vals, A, h->hd, h->he);
    const std::vector<double>& d = h->hd;
    const std::vector<double>& e = h->he;
    for (int64_t i = 0; i < m; i++)
      for (int k = A.rp[i]; k < A.rp[i + 1]; k++) A.v[k] *= e[i] * d[A.ci[k]];
    for (size_t j = 0; j < qdiag.size(); j++) qdiag[j] *= d[j] * d[j];
    if (qcsr.rows)
      for (int64_t i = 0; i < n; i++)
        for (int k = qcsr.rp[i]; k < qcsr.rp[i + 1]; k++) qcsr.v[k] *= d[i] * d[qcsr.ci[k]];
    for (size_t b = 0; b < dia_off.size(); b++)
      for (int64_t i = 0; i + dia_off[b] < n; i++) dia_vals[b][i] *= d[i] * d[i + dia_off[b]];
    for (int64_t j = 0; j < n; j++) {
      hL[j] /= d[j];
      hU[j] /= d[j];
    }
    scale_data(h, hc, hl, hu);
  }

  clk.mark("preconditioning");
  // ---- device problem
  Args& a = h->args;
  std::memset(&a, 0, sizeof(a));
  a.n = n;
  a.m = m;
  a.phi = phi;
  Vec& V = a.V;
  double *dc, *dL, *dU, *dl = nullptr, *du = nullptr;
  if ((st = upload(h, &dc, hc))) return st;
  if ((st = upload(h, &dL, hL))) return st;
  if ((st = upload(h, &dU, hU))) return st;
  if ((st = upload(h, &dl, hl))) return st;
  if ((st = upload(h, &du, hu))) return st;
  V.c = dc;
  V.L = dL;
  V.U = dU;
  V.l = dl;
  V.u = du;
  V.sd = V.se = V.isd = V.ise = nullptr;
  if (h->scaled) {
    std::vector<double> id(n), ie(m);
    for (int64_t j = 0; j < n; j++) id[j] = 1.0 / h->hd[j];
    for (int64_t i = 0; i < m; i++) ie[i] = 1.0 / h->he[i];
    double *p1, *p2, *p3, *p4;
    if ((st = upload(h, &p1, h->hd)) || (st = upload(h, &p2, h->he)) || (st = upload(h, &p3, id)) ||
        (st = upload(h, &p4, ie)))
      return st;
    V.sd = p1;
    V.se = p2;
    V.isd = p3;
    V.ise = p4;
    if ((st = zeros(h, &h->ux, n)) || (st = zeros(h, &h->uy, m)) || (st = zeros(h, &h->uz, n)) ||
        (st = zeros(h, &h->uw, n)))
      return st;
  }
  if (m > 0) {
    if ((st = upload_csr(h, a.A, A))) return st;
    if ((st = upload_transpose(h, a.AT, a.A, A))) return st;
    // SELL copies for the autotuner's choice (not for the persistent mode, which keeps lanes)
    if (h->prm.launch_mode != 3 && h->prm.autotune != 0) {
      if ((st = build_sell_rows(h, a.A)) || (st = build_sell_rows(h, a.AT))) return st;
    }
  } else {
    a.A.cols = n;
    a.AT.cols = 0;
  }
  QDev& QD = a.Q;
  QD.n = n;
  if (!qdiag.empty()) {
    double* d;
    if ((st = upload(h, &d, qdiag))) return st;
    QD.diag = d;
  }
  if (qcsr.rows) {
    if ((st = upload_csr(h, QD.csr, qcsr))) return st;
  }
  if (!dia_off.empty()) {
    QD.ndia = (int)dia_off.size();
    // stored by increasing offset: the main diagonal, if present, comes first (q_local peels it)
    std::vector<int> ord(dia_off.size());
    for (size_t k = 0; k < ord.size(); k++) ord[k] = (int)k;
    std::sort(ord.begin(), ord.end(), [&](int a, int b) { return dia_off[a] < dia_off[b]; });
    std::vector<double> all;
    all.reserve((size_t)QD.ndia * n);
    for (int k = 0; k < QD.ndia; k++) {
      QD.dia_off[k] = dia_off[ord[k]];
      all.insert(all.end(), dia_vals[ord[k]].begin(), dia_vals[ord[k]].end());
    }
    double* d;
    if ((st = upload(h, &d, all))) return st;
    QD.dia = d;
  }
  int64_t toff = 0;
  QD.nfac = (int)facs.size();
  for (int f = 0; f < QD.nfac; f++) {
    if ((st = upload_csr(h, QD.fac[f], facs[f]))) return st;
    if ((st = upload_transpose(h, QD.fact[f], QD.fac[f], facs[f]))) return st;
    QD.toff[f] = toff;
    toff += facs[f].rows;
  }
  QD.ndense = (int)dens.size();
  for (int g = 0; g < QD.ndense; g++) {
    double* d;
    if ((st = upload(h, &d, dens[g].second))) return st;
    QD.dense[g] = d;
    QD.dense_p[g] = dens[g].first;
    QD.toff[QD.nfac + g] = toff;
    toff += dens[g].first;
  }
  QD.tfd = toff;
  if (qap_d) {
    // the QAP product x -> vec(Ahat X Bhat - S X - X T) goes to the intermediate buffers
    // after the factor rows; cuBLAS runs its four DGEMMs on the handle's stream
    double *dq, *tmp, *qin;
    if ((st = upload(h, &dq, qap_vals)) || (st = zeros(h, &tmp, (size_t)qap_d * qap_d)) || (st = zeros(h, &qin, n)))
      return st;
    QD.qap_d = qap_d;
    QD.qap = dq;
    QD.qap_tmp = tmp;
    QD.qap_in = qin;
    QD.qap_off = toff;
    toff += n;
    if ((st = qap_scratch(h, QD))) return st;
  }
  clk.mark("device problem");
  // ---- tiled copies of large factor terms: their one-vector products gather through shared
  // memory (tiled.cu); u = B_f^T B_f x goes to the intermediate buffers at uoff
  {
    int tdev = 0, tsms = 0, optin = 0;
    CU(h, cudaGetDevice(&tdev));
    CU(h, cudaDeviceGetAttribute(&tsms, cudaDevAttrMultiProcessorCount, tdev));
    CU(h, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, tdev));
    const bool room = optin >= (int)(kTileW * sizeof(double)) + 1024;
    bool any = false;
    for (int f = 0; f < QD.nfac; f++) {
      const HostCsr& B = facs[f];
      const int64_t nnz = B.rp[B.rows];
      const int64_t kb = (n + kTileW - 1) / kTileW, kt = (B.rows + kTileW - 1) / kTileW;
      const bool fits = room && h->prm.launch_mode != 3 && kt <= 8 && kb <= kMaxTilesDevice &&
                        kb * B.rows <= ((int64_t)1 << 28);
      const bool large = nnz >= 2000000 && nnz >= 8 * std::max<int64_t>(n, B.rows);
      if (!fits || !(h->prm.tiled_factor == 2 || (h->prm.tiled_factor == 1 && large))) continue;
      if ((st = build_tiled(h, QD.tf[f], QD.fac[f], QD.fact[f], tsms))) return st;
      QD.tiled[f] = 1;
      QD.uoff[f] = toff;
      toff += n;
      any = true;
    }
    if (any) CU(h, tiled_setup());
  }
  // ---- thin factor terms: the inner step forms (B x)_r inside the Q row pass from row r of B.
  // The extra gathers per row of Q are sum_r len(r)^2 / n (every entry of B^T's row j re-reads
  // a whole row of B); at most 1/2 per row the pass saves the pre-pass launch and its latency
  // (S of the n = 1e6 CQP: 1e4 rows of 3, 0.09 per row)
  for (int f = 0; f < QD.nfac; f++) {
    if (QD.tiled[f] || h->prm.factor_inline == 0) continue;
    const HostCsr& B = facs[f];
    double sq = 0.0;
    for (int64_t r = 0; r < B.rows; r++) {
      const double len = (double)(B.rp[r + 1] - B.rp[r]);
      sq += len * len;
    }
    if (h->prm.factor_inline == 2 || sq <= 0.5 * (double)n) QD.inl[f] = 1;
  }
  QD.tlen = toff;

  clk.mark("tiled copies");
  // ---- work vectors (all n- and m-vectors exist; unused ones stay zero)
  double** nvecs[] = {&V.x, &V.w, &V.Qw, &V.ATy, &V.x0, &V.w0, &V.Qw0, &V.ATy0, &V.xb, &V.wb, &V.Qwb, &V.ATyb,
                      &V.wh, &V.Qwh, &V.v, &V.zb, &V.Qxb, &V.xh};
  for (double** p : nvecs)
    if ((st = zeros(h, p, n))) return st;
  double** mvecs[] = {&V.y, &V.y0, &V.yb};
  for (double** p : mvecs)
    if ((st = zeros(h, p, m))) return st;
  if ((st = zeros(h, &V.t1, 2 * std::max<int64_t>(toff, 1)))) return st;
  if ((st = zeros(h, &V.t2, 2 * std::max<int64_t>(toff, 1)))) return st;
  // the autotuner's probe gathers from ain with the column range of every B_f^T (p_f)
  const int64_t nm = std::max(std::max(n, m), toff);
  if ((st = zeros(h, &V.pv, nm))) return st;
  if ((st = zeros(h, &V.pw, nm))) return st;
  if ((st = zeros(h, &V.ptmp, nm))) return st;
  double *ain, *aout;
  if ((st = zeros(h, &ain, nm))) return st;
  if ((st = zeros(h, &aout, nm))) return st;
  V.ain = ain;
  V.aout = aout;

  clk.mark("work vectors");
  // ---- launch plan
  int dev = 0, sms = 0;
  CU(h, cudaGetDevice(&dev));
  CU(h, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->dev = dev;
  Plan& P = h->plan;
  auto chunks = [](int64_t rows) { return (int)std::max<int64_t>(1, (rows + kChunk - 1) / kChunk); };
  const int per_sm = 4;
  P.gridN = std::min(chunks(n), sms * per_sm);
  P.gridM = std::min(chunks(m), sms * per_sm);
  P.gridE = std::min(chunks(n), sms * 8);
  P.gridT = tiled_tbt_grid(n, sms);
  P.gridPre = (int)std::min<int64_t>(std::max<int64_t>(1, (toff + 7) / 8), sms * 8);
  std::function<int(int)> pre_grid;
  {
    // lanes per factor row of the pre-pass: full warps only for long rows (the shuffle
    // reduction costs FP64 instructions that short rows cannot amortise)
    int64_t fnnz = 0, frows = 0;
    for (auto& B : facs) {
      fnnz += B.rp[B.rows];
      frows += B.rows;
    }
    const double avg = frows ? (double)fnnz / (double)frows : 0.0;
    P.gPre = avg < 8 ? 1 : avg < 32 ? 4 : avg < 96 ? 8 : 32;
    // the pre-pass is a grid-stride loop over factor rows: launch only the blocks its rows
    // need (a short factor such as S with 1e4 rows needs 40 blocks, not a full wave)
    int64_t drows = 0;   // dense factor rows take one warp each
    for (auto& F : dens) drows += F.first;
    pre_grid = [frows, drows, sms](int G) {
      return (int)std::min<int64_t>(std::max<int64_t>(1, (frows * G + drows * 32 + kThreads - 1) / kThreads),
                                    (int64_t)sms * 8);
    };
    P.gridPre = pre_grid(P.gPre);
  }
  a.nbM = P.gridM;
  if (h->prm.launch_mode == 3) {
    // persistent solver: one block per row chunk of the larger dimension, at most the
    // co-resident blocks of its kernel
    const int cap = persist_max_blocks(sms);
    if (cap < 1) return fail(h, HPRQP_CUDA_ERROR, "persistent solver: no co-resident blocks");
    P.gridP = (int)std::min<int64_t>(std::max(chunks(n), chunks(std::max<int64_t>(m, 1))), cap);
  }
  const int gmax = std::max(std::max(P.gridN, P.gridM), P.gridP);
  if ((st = zeros(h, &a.partL, (size_t)gmax * kWL))) return st;
  if ((st = zeros(h, &a.part3, (size_t)gmax * kW3))) return st;
  if ((st = zeros(h, &a.partR, (size_t)gmax * kWR))) return st;
  if ((st = zeros(h, &a.partP, (size_t)gmax * kWP))) return st;
  {
    void* p;
    if ((st = dalloc(h, &p, 16 * sizeof(unsigned)))) return st;
    CU(h, cudaMemsetAsync(p, 0, 16 * sizeof(unsigned), h->stream));
    a.counters = (unsigned*)p;
    if ((st = dalloc(h, &p, sizeof(CheckRec) * kHistCap))) return st;
    a.hist = (CheckRec*)p;
    if ((st = dalloc(h, &p, sizeof(Ctrl)))) return st;
    CU(h, cudaMemsetAsync(p, 0, sizeof(Ctrl), h->stream));
    h->dctrl = (Ctrl*)p;
    a.C = h->dctrl;
  }
  CU(h, cudaMallocHost(&h->hctrl, sizeof(Ctrl)));
  std::memset(h->hctrl, 0, sizeof(Ctrl));
  if (a.Q.present() && m > 0) {
    // state of the power method on A A^* when it runs beside the one on Q
    Args& pa = h->pwA_args;
    pa = a;
    void* p;
    if ((st = dalloc(h, &p, sizeof(Ctrl)))) return st;
    CU(h, cudaMemsetAsync(p, 0, sizeof(Ctrl), h->stream));
    h->dctrl2 = (Ctrl*)p;
    pa.C = h->dctrl2;
    if ((st = dalloc(h, &p, 16 * sizeof(unsigned)))) return st;
    CU(h, cudaMemsetAsync(p, 0, 16 * sizeof(unsigned), h->stream));
    pa.counters = (unsigned*)p;
    if ((st = zeros(h, &pa.partP, (size_t)gmax * kWP))) return st;
    if ((st = zeros(h, &pa.V.pv, m))) return st;
    if ((st = zeros(h, &pa.V.pw, m))) return st;
    if ((st = zeros(h, &pa.V.ptmp, n))) return st;
    CU(h, cudaMallocHost(&h->hctrl2, sizeof(Ctrl)));
    std::memset(h->hctrl2, 0, sizeof(Ctrl));
    CU(h, cudaStreamCreateWithFlags(&h->pstream, cudaStreamNonBlocking));
    CU(h, cudaEventCreateWithFlags(&h->pfork, cudaEventDisableTiming));
    CU(h, cudaEventCreateWithFlags(&h->pjoin, cudaEventDisableTiming));
    h->pw_pair = true;
  }
  CU(h, cudaMallocHost(&h->hflags, 8 * sizeof(int)));
  CU(h, cudaEventCreate(&h->ev[0]));
  CU(h, cudaEventCreate(&h->ev[1]));
  CU(h, cudaStreamSynchronize(h->stream));

  clk.mark("launch plan");
  // ---- schedule autotune (lanes per row for each CSR pass)
  {
    CU(h, cudaMemsetAsync(ain, 0, nm * sizeof(double), h->stream));
    P.gA = m > 0 ? tune_G(h, a.A, P.gridM, ain, aout, 1) : 1;
    P.gAT = m > 0 ? tune_G(h, a.AT, P.gridN, ain, aout, 1) : 1;
    const Csr* big = nullptr;
    if (QD.csr.rows) big = &QD.csr;
    for (int f = 0; f < QD.nfac; f++)
      if (!big || QD.fact[f].nnz > big->nnz) big = &QD.fact[f];
    P.gQ = big ? tune_G(h, *big, P.gridN, ain, aout, 1) : 1;
    // Q's CSR-like parts are only thin factors formed on demand: one lane per row (their few
    // entries gain nothing from more lanes, and the bare-SpMV probe cannot see the on-demand
    // products).  A SELL copy of B^T, which packs a chunk's entries into one warp, measured
    // slower on the n = 1e6 CQP (longer chain of dependent loads per entry).
    {
      bool only_inl = QD.nfac > 0 && !QD.csr.rows;
      for (int f = 0; f < QD.nfac; f++) only_inl = only_inl && (QD.tiled[f] || QD.inl[f]);
      if (only_inl && h->prm.autotune == 1) P.gQ = 1;
    }
    bool untiled = false;   // the probe below runs the one-vector pre-pass, which skips tiled terms
    for (int f = 0; f < QD.nfac; f++) untiled = untiled || !QD.tiled[f];
    if (QD.nfac > 0 && h->prm.autotune == 1 && untiled) {
      // lanes per factor row of the pre-pass, timed on the pre-pass itself
      float best = 1e30f;
      for (int G : {1, 4, 8, 32}) {
        const int grid = pre_grid(G);
        CU(h, launch_pre_probe(a, G, grid, h->stream));
        CU(h, cudaEventRecord(h->ev[0], h->stream));
        for (int r = 0; r < 3; r++) CU(h, launch_pre_probe(a, G, grid, h->stream));
        CU(h, cudaEventRecord(h->ev[1], h->stream));
        CU(h, cudaEventSynchronize(h->ev[1]));
        float ms = 0;
        CU(h, cudaEventElapsedTime(&ms, h->ev[0], h->ev[1]));
        if (ms < best) {
          best = ms;
          P.gPre = G;
          P.gridPre = grid;
        }
      }
    }
    CU(h, cudaStreamSynchronize(h->stream));
    CU(h, cudaGetLastError());
    CU(h, plan_plain_grids(a, P, sms));
    // plain steps of the fixed-schedule graph end with the fused passes (need Q and A)
    P.fuse = (h->prm.fused_steps != 0 && QD.present() && m > 0) ? 1 : 0;
  }
  clk.mark("autotune");
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_create(hprqp_handle** out, int64_t n, int64_t m, const hprqp_qop* Q,
                                     const int32_t* A_rowptr, const int32_t* A_colidx, const double* A_vals,
                                     const double* c, const double* l, const double* u, const double* L,
                                     const double* U, int32_t phi, double lambda, const hprqp_params* params) {
  g_create_err.clear();
  if (!out) return fail(nullptr, HPRQP_INVALID_ARG, "null handle pointer");
  *out = nullptr;
  hprqp_handle* h = new hprqp_handle();
  if (params) h->prm = *params;
  else hprqp_default_params(&h->prm);
  if (h->prm.check_every < 1 || h->prm.restart_every < 1 || h->prm.iters_per_launch < 1 ||
      h->prm.iters_per_launch > 4096 || h->prm.launch_mode < 0 || h->prm.launch_mode > 3 || h->prm.method < 0 ||
      h->prm.method > 2) {
    fail(nullptr, HPRQP_INVALID_ARG,
         "check_every, restart_every >= 1, 1 <= iters_per_launch <= 4096, launch_mode 0..3, method 0..2");
    delete h;
    return HPRQP_INVALID_ARG;
  }
  if (h->prm.stream) {
    h->stream = (cudaStream_t)h->prm.stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      fail(nullptr, HPRQP_CUDA_ERROR, "cannot create a CUDA stream (no device?)");
      delete h;
      return HPRQP_CUDA_ERROR;
    }
    h->own_stream = true;
  }
  hprqp_status st;
  {
    Range r("hprqp_create");
    st = create_impl(h, n, m, Q, A_rowptr, A_colidx, A_vals, c, l, u, L, U, phi, lambda);
  }
  if (st != HPRQP_OK) {
    if (g_create_err.empty()) g_create_err = h->err;
    release(h);
    return st;
  }
  *out = h;
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ warm start
extern "C" hprqp_status hprqp_set_warm_start(hprqp_handle* h, const double* x0, const double* y0, double sigma0) {
  if (!h) return HPRQP_INVALID_ARG;
  hprqp_status st;
  // validate into temporaries: a rejected warm start leaves the previous one in place
  std::vector<double> wx, wy;
  if (x0) {
    if ((st = fetch(h, wx, x0, h->n))) return st;
    for (double v : wx)
      if (!std::isfinite(v)) return fail(h, HPRQP_INVALID_ARG, "warm start x0 is not finite");
  }
  if (y0 && h->m > 0) {
    if ((st = fetch(h, wy, y0, h->m))) return st;
    for (double v : wy)
      if (!std::isfinite(v)) return fail(h, HPRQP_INVALID_ARG, "warm start y0 is not finite");
  }
  h->ws_x.swap(wx);
  h->ws_y.swap(wy);
  h->ws_sigma = sigma0 > 0 && std::isfinite(sigma0) ? sigma0 : 0.0;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_set_data(hprqp_handle* h, const double* c, const double* l, const double* u) {
  if (!h) return HPRQP_INVALID_ARG;
  hprqp_status st;
  Vec& V = h->args.V;
  const int64_t n = h->n, m = h->m;
  std::vector<double> hc, hl, hu;
  if ((st = fetch(h, hc, c ? c : V.c, n))) return st;
  if ((st = fetch(h, hl, l ? l : V.l, m))) return st;
  if ((st = fetch(h, hu, u ? u : V.u, m))) return st;
  if (h->scaled) {   // the kept pieces are stored scaled: back to the original data first
    if (!c)
      for (int64_t j = 0; j < n; j++) hc[j] /= h->hd[j];
    if (!l)
      for (int64_t i = 0; i < m; i++) hl[i] /= h->he[i];
    if (!u)
      for (int64_t i = 0; i < m; i++) hu[i] /= h->he[i];
  }
  const double nb2 = h->nb2, nc2 = h->nc2, bi = h->b_inf, ci = h->c_inf;
  if ((st = data_norms(h, hc, hl, hu))) {
    h->nb2 = nb2;
    h->nc2 = nc2;
    h->b_inf = bi;
    h->c_inf = ci;
    return st;
  }
  if (h->scaled) scale_data(h, hc, hl, hu);
  if (c) CU(h, cudaMemcpyAsync((void*)V.c, hc.data(), n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (l && m) CU(h, cudaMemcpyAsync((void*)V.l, hl.data(), m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  if (u && m) CU(h, cudaMemcpyAsync((void*)V.u, hu.data(), m * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  h->solved = false;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_set_wait_polls(hprqp_handle* h, int32_t polls) {
  if (!h) return HPRQP_INVALID_ARG;
  if (polls < 0) return fail(h, HPRQP_INVALID_ARG, "wait_polls must be >= 0");
  h->prm.wait_polls = polls;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_set_lambda(hprqp_handle* h, double lambda_A, double lambda_Q) {
  if (!h) return HPRQP_INVALID_ARG;
  if (!(lambda_A >= 0.0 && std::isfinite(lambda_A)) || !(lambda_Q >= 0.0 && std::isfinite(lambda_Q)))
    return fail(h, HPRQP_INVALID_ARG, "lambda_A and lambda_Q must be finite and >= 0");
  h->prm.lambda_A = lambda_A;
  h->prm.lambda_Q = lambda_Q;
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ graphs
// The fixed-schedule graph (used while at least fixed_L iterations remain): L = lcm of the
// R~-test and stopping-test periods, at most 1024 steps; left out when larger or when the
// driver rejects it (the dynamic graph then runs every step).
static void build_fixed(hprqp_handle* h) {
  if (h->fixed_tried) return;
  h->fixed_tried = true;
  if (h->prm.launch_mode != 0 || !h->prm.fixed_schedule) return;
  if (!h->side && cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  const int64_t ce = h->prm.check_every, re = h->prm.restart_off ? ce : h->prm.restart_every;
  int64_t a = re, b = ce;
  while (b) {
    const int64_t t = a % b;
    a = b;
    b = t;
  }
  const int64_t L = re / a * ce;
  if (L > 1024) return;
  // with programmatic launches first; without them if the driver rejects that graph
  for (int attempt = 0; attempt < 2; attempt++) {
    if (attempt == 1 && !h->prm.pdl) break;
    h->plan.pdl = attempt == 0 && h->prm.pdl ? 1 : 0;
    cudaGraph_t g;
    if (build_fixed_graph(h->args, h->plan, h->stream, h->side, (int)L, (int)re, (int)ce, &g, &h->fixed_kernels) !=
        cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaError_t ie = cudaGraphInstantiate(&h->g_fixed, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
      cudaGetLastError();
      h->g_fixed = nullptr;
      continue;
    }
    h->fixed_L = (int)L;
    h->conditional = true;   // conditional nodes work on this device
    return;
  }
  h->plan.pdl = 0;
}

static hprqp_status build_iter_graph(hprqp_handle* h) {
  if (h->g_iter) return HPRQP_OK;
  cudaGraph_t g;
  // preferred: device-selected step variants through conditional nodes
  if (!h->side) CU(h, cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking));
  // with programmatic launches first; without them if the driver rejects that graph
  for (int attempt = 0; attempt < 2 && h->prm.launch_mode == 0; attempt++) {
    h->plan.pdl = attempt == 0 && h->prm.pdl ? 1 : 0;
    if (attempt == 1 && !h->prm.pdl) break;
    cudaError_t be = build_conditional_graph(h->args, h->plan, h->stream, h->side, h->prm.iters_per_launch, &g);
    if (be == cudaSuccess) {
      cudaError_t ie = cudaGraphInstantiate(&h->g_iter, g, 0);
      cudaGraphDestroy(g);
      if (ie == cudaSuccess) {
        h->conditional = true;
        return HPRQP_OK;
      }
      h->g_iter = nullptr;
    }
    cudaGetLastError();
  }
  h->plan.pdl = 0;
  cudaGetLastError();
  // fallback: every kernel launched each step, variants decided inside the kernels
  h->conditional = false;
  CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < h->prm.iters_per_launch && le == cudaSuccess; i++) {
    le = launch_iteration(h->args, h->plan, h->stream);
    if (le == cudaSuccess) le = launch_restart(h->args, h->plan, h->stream);
  }
  cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    cudaGetLastError();
    if (ce == cudaSuccess) cudaGraphDestroy(g);
    return fail(h, HPRQP_CUDA_ERROR, "graph capture failed: %s / %s", cudaGetErrorString(le), cudaGetErrorString(ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&h->g_iter, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    h->g_iter = nullptr;
    return fail(h, HPRQP_CUDA_ERROR, "graph instantiate failed: %s", cudaGetErrorString(ie));
  }
  return HPRQP_OK;
}

// The arguments of the power method on A A^* when it runs beside the one on Q: the solver's,
// with its own controller copy, partials, counters and vectors.
static Args pw_pair_args(const hprqp_handle* h) {
  Args pa = h->args;
  pa.C = h->pwA_args.C;
  pa.counters = h->pwA_args.counters;
  pa.partP = h->pwA_args.partP;
  pa.V.pv = h->pwA_args.V.pv;
  pa.V.pw = h->pwA_args.V.pw;
  pa.V.ptmp = h->pwA_args.V.ptmp;
  return pa;
}

static hprqp_status build_pw_graph(hprqp_handle* h, int which) {
  if (h->g_pw[which]) return HPRQP_OK;
  const Args pa = (which == 0 && h->pw_pair) ? pw_pair_args(h) : h->args;
  cudaGraph_t g;
  CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  // an even number of iterations per graph, so that every launch starts reading pv
  for (int i = 0; i < h->pw_chunk && le == cudaSuccess; i++) le = launch_power_iter(pa, h->plan, which, i, h->stream);
  cudaError_t ce = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess || ce != cudaSuccess) {
    cudaGetLastError();
    if (ce == cudaSuccess) cudaGraphDestroy(g);
    return fail(h, HPRQP_CUDA_ERROR, "power graph capture failed");
  }
  cudaError_t ie = cudaGraphInstantiate(&h->g_pw[which], g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    h->g_pw[which] = nullptr;
    return fail(h, HPRQP_CUDA_ERROR, "power graph instantiate failed");
  }
  return HPRQP_OK;
}

// Power method of Sec. 4.1 on A A^* (which = 0, R^m) or Q (which = 1, R^n); returns the
// Rayleigh quotient at convergence times the safety factor.
static hprqp_status power_method(hprqp_handle* h, int which, double* lam) {
  Range rg(which == 0 ? "hprqp_power_A" : "hprqp_power_Q");
  const int64_t dim = which == 0 ? h->m : h->n;
  hprqp_status st;
  if ((st = build_pw_graph(h, which))) return st;
  // host value of 1/||start||, same start vector and summation order as the CPU reference
  double s2 = 0.0;
  for (int64_t i = 0; i < dim; i++) {
    uint32_t hh = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
    double v = 0.5 + (double)hh / 4294967296.0;
    s2 += v * v;
  }
  // with the paired state (m > 0 and Q present), the method on A A^* keeps to its own
  // controller copy and vectors, as its graph does, also when it runs alone
  const bool pair = which == 0 && h->pw_pair;
  Ctrl* hc = pair ? h->hctrl2 : h->hctrl;
  Ctrl* dc = pair ? h->dctrl2 : h->dctrl;
  if (pair) std::memcpy(hc, h->hctrl, sizeof(Ctrl));
  Ctrl& C = *hc;
  C.pw_it = 0;
  C.pw_lam = 0.0;
  C.pw_done = 0;
  C.pw_scale = 1.0 / std::sqrt(s2);
  C.pw_max = h->prm.power_max_iter;
  C.pw_tol = h->prm.power_tol;
  C.done = 1;  // keep the iteration kernels idle
  CU(h, cudaMemcpyAsync(dc, hc, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  CU(h, launch_power_init(pair ? pw_pair_args(h) : h->args, h->plan, which, h->stream));
  const int64_t max_launch = h->prm.power_max_iter / h->pw_chunk + 3;
  int* flag = h->hflags;
  h->launches += 1;
  const int64_t pw_nodes = (int64_t)h->pw_chunk * kernels_per_power_iter(h->args, which);
  for (int64_t i = 0; i < max_launch; i++) {
    CU(h, cudaGraphLaunch(h->g_pw[which], h->stream));
    h->launches += pw_nodes;
    CU(h, cudaMemcpyAsync(flag, &dc->pw_done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (*flag == 1) break;
  }
  CU(h, cudaMemcpyAsync(hc, dc, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  *lam = h->prm.power_safety * hc->pw_lam;
  return HPRQP_OK;
}

// Both power methods of Sec. 4.1 at once (m > 0 and Q present): the one on Q on the solver's
// stream, the one on A A^* on its own stream with its own state, each chunk of iterations a
// graph launch; the host polls both done flags after every round of launches.  The two are
// independent and each product leaves most of the GPU's issue slots idle, so they overlap.
static hprqp_status power_both(hprqp_handle* h, double* lamA, double* lamQ) {
  Range rg("hprqp_power_AQ");
  hprqp_status st;
  if ((st = build_pw_graph(h, 0))) return st;
  if ((st = build_pw_graph(h, 1))) return st;
  const Args pa = pw_pair_args(h);
  auto start_scale = [](int64_t dim) {
    // host value of 1/||start||, same start vector and summation order as the CPU reference
    double s2 = 0.0;
    for (int64_t i = 0; i < dim; i++) {
      uint32_t hh = (uint32_t)((uint64_t)(i + 1) * 2654435761u);
      double v = 0.5 + (double)hh / 4294967296.0;
      s2 += v * v;
    }
    return 1.0 / std::sqrt(s2);
  };
  Ctrl* hc[2] = {h->hctrl2, h->hctrl};
  Ctrl* dc[2] = {h->dctrl2, h->dctrl};
  cudaStream_t ss[2] = {h->pstream, h->stream};
  CU(h, cudaEventRecord(h->pfork, h->stream));
  CU(h, cudaStreamWaitEvent(h->pstream, h->pfork, 0));
  for (int w = 0; w < 2; w++) {
    Ctrl& C = *hc[w];
    if (w == 0) std::memcpy(&C, h->hctrl, sizeof(Ctrl));
    C.pw_it = 0;
    C.pw_lam = 0.0;
    C.pw_done = 0;
    C.pw_scale = start_scale(w == 0 ? h->m : h->n);
    C.pw_max = h->prm.power_max_iter;
    C.pw_tol = h->prm.power_tol;
    C.done = 1;  // keep the iteration kernels idle
    CU(h, cudaMemcpyAsync(dc[w], hc[w], sizeof(Ctrl), cudaMemcpyHostToDevice, ss[w]));
    CU(h, launch_power_init(w == 0 ? pa : h->args, h->plan, w, ss[w]));
    h->launches += 1;
  }
  const int64_t max_launch = h->prm.power_max_iter / h->pw_chunk + 3;
  int* flag = h->hflags + 2;
  bool done[2] = {false, false};
  for (int64_t i = 0; i < max_launch && !(done[0] && done[1]); i++) {
    for (int w = 0; w < 2; w++) {
      if (done[w]) continue;
      CU(h, cudaGraphLaunch(h->g_pw[w], ss[w]));
      h->launches += (int64_t)h->pw_chunk * kernels_per_power_iter(h->args, w);
      CU(h, cudaMemcpyAsync(flag + w, &dc[w]->pw_done, sizeof(int), cudaMemcpyDeviceToHost, ss[w]));
    }
    for (int w = 0; w < 2; w++) {
      if (done[w]) continue;
      CU(h, cudaStreamSynchronize(ss[w]));
      done[w] = flag[w] == 1;
    }
  }
  for (int w = 0; w < 2; w++) CU(h, cudaMemcpyAsync(hc[w], dc[w], sizeof(Ctrl), cudaMemcpyDeviceToHost, ss[w]));
  CU(h, cudaEventRecord(h->pjoin, h->pstream));
  CU(h, cudaStreamWaitEvent(h->stream, h->pjoin, 0));
  CU(h, cudaStreamSynchronize(h->stream));
  CU(h, cudaStreamSynchronize(h->pstream));
  *lamA = h->prm.power_safety * h->hctrl2->pw_lam;
  *lamQ = h->prm.power_safety * h->hctrl->pw_lam;
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ solve
// Starting point u^{0,0} (origin or warm start, w = x), its images, and the controller state.
static hprqp_status init_state(hprqp_handle* h, double lamA, double lamQ, double sigma, double tol, int64_t max_iter) {
  Args& a = h->args;
  const bool HQ = a.Q.present(), HA = h->m > 0;
  Vec& V = a.V;
  const size_t nb8 = h->n * sizeof(double), mb8 = h->m * sizeof(double);
  if (!h->ws_x.empty()) {
    CU(h, cudaMemcpyAsync(V.x, h->ws_x.data(), nb8, cudaMemcpyHostToDevice, h->stream));
  } else {
    CU(h, cudaMemsetAsync(V.x, 0, nb8, h->stream));
  }
  if (h->scaled && !h->ws_x.empty()) CU(h, launch_vmul(V.x, V.isd, h->n, h->stream));   // xs = D^{-1} x0
  CU(h, cudaMemcpyAsync(V.w, V.x, nb8, cudaMemcpyDeviceToDevice, h->stream));
  CU(h, cudaMemcpyAsync(V.x0, V.x, nb8, cudaMemcpyDeviceToDevice, h->stream));
  CU(h, cudaMemcpyAsync(V.w0, V.x, nb8, cudaMemcpyDeviceToDevice, h->stream));
  if (HA) {
    if (!h->ws_y.empty()) CU(h, cudaMemcpyAsync(V.y, h->ws_y.data(), mb8, cudaMemcpyHostToDevice, h->stream));
    else CU(h, cudaMemsetAsync(V.y, 0, mb8, h->stream));
    if (h->scaled && !h->ws_y.empty()) CU(h, launch_vmul(V.y, V.ise, h->m, h->stream));   // ys = E^{-1} y0
    CU(h, cudaMemcpyAsync(V.y0, V.y, mb8, cudaMemcpyDeviceToDevice, h->stream));
  }
  // images Q w^0 and A^* y^0
  if (HQ) {
    if (!h->ws_x.empty()) {
      CU(h, cudaMemcpyAsync((void*)V.ain, V.x, nb8, cudaMemcpyDeviceToDevice, h->stream));
      CU(h, launch_apply(a, h->plan, 2, h->stream));
      h->launches += 1 + (a.Q.has_pre() ? 1 : 0);
      CU(h, cudaMemcpyAsync(V.Qw, V.aout, nb8, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CU(h, cudaMemsetAsync(V.Qw, 0, nb8, h->stream));
    }
    CU(h, cudaMemcpyAsync(V.Qw0, V.Qw, nb8, cudaMemcpyDeviceToDevice, h->stream));
  }
  if (HA) {
    if (!h->ws_y.empty()) {
      CU(h, cudaMemcpyAsync((void*)V.ain, V.y, mb8, cudaMemcpyDeviceToDevice, h->stream));
      CU(h, launch_apply(a, h->plan, 1, h->stream));
      h->launches += 1;
      CU(h, cudaMemcpyAsync(V.ATy, V.aout, nb8, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      CU(h, cudaMemsetAsync(V.ATy, 0, nb8, h->stream));
    }
    CU(h, cudaMemcpyAsync(V.ATy0, V.ATy, nb8, cudaMemcpyDeviceToDevice, h->stream));
  }
  CU(h, cudaMemsetAsync(a.counters, 0, 16 * sizeof(unsigned), h->stream));
  Ctrl& C = *h->hctrl;
  std::memset(&C, 0, sizeof(Ctrl));
  C.lamA = lamA;
  C.lamQ = lamQ;
  C.lambda = h->lambda;
  C.tol = tol;
  C.alpha1 = h->prm.alpha1;
  C.alpha2 = h->prm.alpha2;
  C.alpha3 = h->prm.alpha3;
  C.alpha3_tight = h->prm.alpha3_tight;
  C.ratio_tight = h->prm.ratio_tight;
  C.c_inf = h->c_inf;
  C.b_inf = h->b_inf;
  C.max_iter = max_iter;
  C.check_every = h->prm.check_every;
  C.restart_every = h->prm.restart_every;
  C.halpern_total = h->prm.halpern_total;
  C.restart_off = h->prm.restart_off;
  C.sigma_fixed = h->prm.sigma_fixed;
  C.sigma_golden = h->prm.sigma_golden;
  C.has_A = HA;
  C.has_Q = HQ;
  C.phi = h->phi;
  C.mode = 0;
  C.k = C.t = C.r = 0;
  C.R_first = -1.0;
  C.rtest = !C.restart_off;
  C.ttest = (1 % C.check_every == 0) || (1 >= max_iter);
  C.status = 1;
  C.done = 0;
  C.pw_done = 1;
  hprqp::set_sigma(C, sigma);
  halpern_weights(C, C.fha, C.fhb);
  CU(h, cudaMemcpyAsync(h->dctrl, h->hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, h->stream));
  return HPRQP_OK;
}

static double initial_sigma(hprqp_handle* h) {
  if (h->ws_sigma > 0) return h->ws_sigma;
  if (h->prm.sigma0 > 0) return h->prm.sigma0;
  // Sec. 4.1: sigma0 = ||b|| / ||c|| when both lie in [1e-16, 1e16], else 1
  double nb = std::sqrt(h->nb2), nc = std::sqrt(h->nc2);
  return (nb >= 1e-16 && nb <= 1e16 && nc >= 1e-16 && nc <= 1e16) ? nb / nc : 1.0;
}

static hprqp_status finish_solve(hprqp_handle* h, std::chrono::steady_clock::time_point t0,
                                 std::chrono::steady_clock::time_point t1, double lamA, double lamQ, double sigma,
                                 bool time_up);

// launch_mode 2: the same step variants as the conditional graph, launched one step at a time
// on the stream, the host reading the controller state after each step.
static hprqp_status solve_stream(hprqp_handle* h, std::chrono::steady_clock::time_point t0,
                                 std::chrono::steady_clock::time_point t1, double lamA, double lamQ, double sigma) {
  Ctrl& C = *h->hctrl;
  bool time_up = false;
  for (;;) {
    const int var = C.done ? 3 : C.ttest ? 2 : C.rtest ? 1 : 0;
    if (var == 3) break;
    CU(h, launch_step_var(h->args, h->plan, h->stream, var));
    CU(h, cudaMemcpyAsync(h->hctrl, h->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (C.restart_pending && !C.done) {
      CU(h, launch_restart(h->args, h->plan, h->stream));
      CU(h, cudaMemcpyAsync(h->hctrl, h->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
      CU(h, cudaStreamSynchronize(h->stream));
    }
    if (h->prm.time_limit > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > h->prm.time_limit) {
      time_up = true;
      break;
    }
  }
  return finish_solve(h, t0, t1, lamA, lamQ, sigma, time_up);
}


// ------------------------------------------------------------------------------------ primal HPR
// Appendix A, Algorithms 6 (method 1) and 7 (method 2); see primal.cu for the steps.
static hprqp_status primal_alloc(hprqp_handle* h) {
  if (h->primal_ready) return HPRQP_OK;
  const int64_t n = h->n, m = h->m;
  hprqp_status st;
  double** nv[] = {&h->px, &h->pv, &h->pt, &h->px0, &h->pv0, &h->pt0, &h->pxb, &h->pvb, &h->ptb, &h->pzb,
                   &h->pQv, &h->pATw, &h->pQxb, &h->pATyb};
  for (double** q : nv)
    if ((st = zeros(h, q, n))) return st;
  double** mv[] = {&h->ps, &h->py, &h->ps0, &h->py0, &h->psb, &h->pyb, &h->pAx, &h->pw, &h->pAxb};
  for (double** q : mv)
    if ((st = zeros(h, q, m))) return st;
  if ((st = zeros(h, &h->ppn, (size_t)primal_eta_blocks(n) * 8))) return st;
  if ((st = zeros(h, &h->ppm, (size_t)primal_eta_blocks(std::max<int64_t>(m, 1)) * 4))) return st;
  if ((st = zeros(h, &h->pout, 8))) return st;
  h->primal_ready = true;
  return HPRQP_OK;
}

// out = op(in) through the solver's operator kernels (op 0: A, 1: A^T, 2: Q)
static hprqp_status primal_apply(hprqp_handle* h, int op, const double* in, double* out, int64_t& launches) {
  Vec& V = h->args.V;
  const int64_t nin = op == 1 ? h->m : h->n, nout = op == 0 ? h->m : h->n;
  CU(h, cudaMemcpyAsync((void*)V.ain, in, nin * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  CU(h, launch_apply(h->args, h->plan, op, h->stream));
  CU(h, cudaMemcpyAsync(out, V.aout, nout * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  launches += 1 + (op == 2 && h->args.Q.has_pre() ? 1 : 0);
  return HPRQP_OK;
}

static hprqp_status solve_primal(hprqp_handle* h, double tol, int64_t max_iter, std::chrono::steady_clock::time_point t0,
                                 std::chrono::steady_clock::time_point t1, double lamA, double lamQ) {
  hprqp_status st;
  if ((st = primal_alloc(h))) return st;
  Args& a = h->args;
  Vec& V = a.V;
  const int64_t n = h->n, m = h->m;
  const bool HQ = a.Q.present(), HA = m > 0, two = h->prm.method == 2;
  const double sigma = initial_sigma(h);
  const double tau = two ? sigma * (1.0 + lamA) : lamQ + sigma * lamA;
  const size_t nb8 = n * sizeof(double), mb8 = m * sizeof(double);
  cudaStream_t s = h->stream;
  int64_t L = 0;
  // starting point: x = v = x0 (warm start or origin), y = y0, s = t = 0
  if (!h->ws_x.empty()) CU(h, cudaMemcpyAsync(h->px, h->ws_x.data(), nb8, cudaMemcpyHostToDevice, s));
  else CU(h, cudaMemsetAsync(h->px, 0, nb8, s));
  CU(h, cudaMemcpyAsync(h->pv, h->px, nb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaMemsetAsync(h->pt, 0, nb8, s));
  if (HA) {
    if (!h->ws_y.empty()) CU(h, cudaMemcpyAsync(h->py, h->ws_y.data(), mb8, cudaMemcpyHostToDevice, s));
    else CU(h, cudaMemsetAsync(h->py, 0, mb8, s));
    CU(h, cudaMemsetAsync(h->ps, 0, mb8, s));
    CU(h, cudaMemcpyAsync(h->py0, h->py, mb8, cudaMemcpyDeviceToDevice, s));
    CU(h, cudaMemsetAsync(h->ps0, 0, mb8, s));
    CU(h, cudaMemsetAsync(h->pATw, 0, nb8, s));
  } else {
    CU(h, cudaMemsetAsync(h->pATw, 0, nb8, s));
    CU(h, cudaMemsetAsync(h->pATyb, 0, nb8, s));
  }
  CU(h, cudaMemcpyAsync(h->px0, h->px, nb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaMemcpyAsync(h->pv0, h->pv, nb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaMemsetAsync(h->pt0, 0, nb8, s));
  if (!HQ) {
    CU(h, cudaMemsetAsync(h->pQv, 0, nb8, s));
    CU(h, cudaMemsetAsync(h->pQxb, 0, nb8, s));
  }
  double out[5] = {INFINITY, INFINITY, INFINITY, NAN, NAN};
  int status = HPRQP_MAX_ITER;
  int64_t k = 0, k14 = 0, k16 = 0;
  double s14 = 0.0, s16 = 0.0;
  bool time_up = false;
  for (;;) {
    if (HA && (st = primal_apply(h, 0, h->px, h->pAx, L))) return st;
    if (HQ && (st = primal_apply(h, 2, two ? h->pv : h->px, h->pQv, L))) return st;
    if (HA) {
      CU(h, primal_rows(h->pAx, h->py, V.l, V.u, sigma, m, h->psb, h->pyb, h->pw, s));
      L++;
      if ((st = primal_apply(h, 1, h->pw, h->pATw, L))) return st;
    }
    if (two) {
      CU(h, primal_vt(h->pv, h->pQv, h->px, h->pt, lamQ, sigma, n, h->pvb, h->ptb, s));
      L++;
    }
    CU(h, primal_x(h->px, h->pQv, V.c, h->pATw, h->pvb, h->ptb, V.L, V.U, h->phi, h->lambda, sigma, tau, two ? 1 : 0,
                   n, h->pxb, h->pzb, s));
    L++;
    const int64_t kd = k + 1;
    if (kd % h->prm.check_every == 0 || kd >= max_iter) {
      if (HA && (st = primal_apply(h, 0, h->pxb, h->pAxb, L))) return st;
      if (HQ && (st = primal_apply(h, 2, h->pxb, h->pQxb, L))) return st;
      if (HA && (st = primal_apply(h, 1, h->pyb, h->pATyb, L))) return st;
      CU(h, primal_eta(h->pxb, h->pQxb, h->pATyb, h->pzb, h->pAxb, h->pyb, a, h->b_inf, h->c_inf, h->lambda, h->ppn,
                       h->ppm, h->pout, s));
      L += HA ? 3 : 2;
      CU(h, cudaMemcpyAsync(out, h->pout, 5 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CU(h, cudaStreamSynchronize(s));
      const double rk = std::max(out[0], std::max(out[1], out[2]));
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (std::isnan(out[0]) || std::isnan(out[1]) || std::isnan(out[2]) || std::isinf(out[3]) || std::isinf(out[4])) {
        status = HPRQP_NUMERICAL_ERROR;
        k = kd;
        break;
      }
      if (!k14 && rk <= 1e-4) {
        k14 = kd;
        s14 = el;
      }
      if (!k16 && rk <= 1e-6) {
        k16 = kd;
        s16 = el;
      }
      if (rk <= tol) {
        status = HPRQP_OK;
        k = kd;
        break;
      }
      if (kd >= max_iter) {
        k = kd;
        break;
      }
      if (h->prm.time_limit > 0 && el > h->prm.time_limit) {
        status = HPRQP_TIME_LIMIT;
        time_up = true;
        k = kd;
        break;
      }
    }
    // Steps 4-5
    const double ha = 1.0 / (k + 2.0), hb = (k + 1.0) / (k + 2.0);
    {
      double* u[3] = {h->px, h->pv, h->pt};
      const double* u0[3] = {h->px0, h->pv0, h->pt0};
      const double* ub[3] = {h->pxb, h->pvb, h->ptb};
      CU(h, primal_halpern(u, u0, ub, two ? 3 : 1, ha, hb, n, s));
      L++;
    }
    if (HA) {
      double* u[3] = {h->ps, h->py, nullptr};
      const double* u0[3] = {h->ps0, h->py0, nullptr};
      const double* ub[3] = {h->psb, h->pyb, nullptr};
      CU(h, primal_halpern(u, u0, ub, 2, ha, hb, m, s));
      L++;
    }
    k = kd;
  }
  (void)time_up;
  // the output of the last iteration goes where hprqp_get reads it
  CU(h, cudaMemcpyAsync(V.xb, h->pxb, nb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaMemcpyAsync(V.zb, h->pzb, nb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaMemcpyAsync(V.wb, two ? h->pvb : h->pxb, nb8, cudaMemcpyDeviceToDevice, s));
  if (HA) CU(h, cudaMemcpyAsync(V.yb, h->pyb, mb8, cudaMemcpyDeviceToDevice, s));
  CU(h, cudaStreamSynchronize(s));
  auto t2 = std::chrono::steady_clock::now();
  hprqp_kkt& K = h->kkt;
  std::memset(&K, 0, sizeof(K));
  K.lanes_q = h->plan.gQ;
  K.lanes_a = h->plan.gA;
  K.lanes_at = h->plan.gAT;
  K.lanes_pre = h->plan.gPre;
  for (int f = 0; f < h->args.Q.nfac; f++) K.tiled_terms += h->args.Q.tiled[f];
  K.eta_p = out[0];
  K.eta_d = out[1];
  K.eta_gap = out[2];
  K.rel_kkt = std::max(out[0], std::max(out[1], out[2]));
  K.pobj = out[3];
  K.dobj = out[4];
  K.iters = k;
  K.restarts = 0;
  K.sigma = sigma;
  K.lambda_A = lamA;
  K.lambda_Q = lamQ;
  K.solve_seconds = std::chrono::duration<double>(t2 - t0).count();
  K.power_seconds = std::chrono::duration<double>(t1 - t0).count();
  h->launches += L;
  K.kernel_launches = h->launches;
  K.status = status;
  K.iters_1e4 = k14;
  K.iters_1e6 = k16;
  K.seconds_1e4 = s14;
  K.seconds_1e6 = s16;
  h->last_status = status;
  h->solved = true;
  h->last_lamA = lamA;
  h->last_lamQ = lamQ;
  h->last_sigma0 = sigma;
  return (hprqp_status)status;
}

// launch_mode 3: every pass of many inner steps in one cooperative launch (persist.cu);
// the host checks the done flag (and the time limit) between launches.
static hprqp_status solve_persist(hprqp_handle* h, std::chrono::steady_clock::time_point t0,
                                  std::chrono::steady_clock::time_point t1, double lamA, double lamQ, double sigma) {
  Args& a = h->args;
  unsigned* bar = a.counters + 8;
  int* err = reinterpret_cast<int*>(a.counters + 10);
  const long long per = 4096;
  bool time_up = false;
  for (;;) {
    CU(h, launch_persist(a, h->plan, h->plan.gridP, per, bar, err, (unsigned)h->prm.wait_polls, h->stream));
    h->launches += 1;
    CU(h, cudaMemcpyAsync(h->hflags, &h->dctrl->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaMemcpyAsync(h->hflags + 1, err, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    if (h->hflags[1]) return fail(h, HPRQP_TIMEOUT, "persistent solver: a grid barrier wait gave up");
    if (h->hflags[0]) break;
    if (h->prm.time_limit > 0 &&
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > h->prm.time_limit) {
      time_up = true;
      break;
    }
  }
  return finish_solve(h, t0, t1, lamA, lamQ, sigma, time_up);
}

extern "C" hprqp_status hprqp_solve(hprqp_handle* h, double tol, int64_t max_iter) {
  if (!h) return HPRQP_INVALID_ARG;
  h->err.clear();
  if (!(tol > 0.0) || max_iter < 1) return fail(h, HPRQP_INVALID_ARG, "need tol > 0 and max_iter >= 1");
  auto t0 = std::chrono::steady_clock::now();
  hprqp_status st;
  Args& a = h->args;
  const bool HQ = a.Q.present(), HA = h->m > 0;
  CU(h, cudaSetDevice(h->dev));
  h->launches = 0;
  h->fixed_steps = 0;
  // ---- lambda_A >= lambda_1(AA^*), lambda_Q >= lambda_1(Q) (Sec. 4.1)
  double lamA = 0.0, lamQ = 0.0;
  if (HA && HQ && h->pw_pair && !(h->prm.lambda_A > 0) && !(h->prm.lambda_Q > 0)) {
    if ((st = power_both(h, &lamA, &lamQ))) return st;
    if (!(lamA > 0.0)) lamA = 1.0;
  } else {
    if (HA) {
      if (h->prm.lambda_A > 0) lamA = h->prm.lambda_A;
      else if ((st = power_method(h, 0, &lamA))) return st;
      if (!(lamA > 0.0)) lamA = 1.0;
    }
    if (HQ) {
      if (h->prm.lambda_Q > 0) lamQ = h->prm.lambda_Q;
      else if ((st = power_method(h, 1, &lamQ))) return st;
    }
  }
  auto t1 = std::chrono::steady_clock::now();
  if (h->prm.method != 0) {
    if (h->scaled) return fail(h, HPRQP_INVALID_ARG, "the primal methods run without preconditioning: create with scaling = 0");
    return solve_primal(h, tol, max_iter, t0, t1, lamA, lamQ);
  }
  const double sigma = initial_sigma(h);
  if ((st = init_state(h, lamA, lamQ, sigma, tol, max_iter))) return st;
  CU(h, launch_stamp(a, h->stream));
  h->launches += 1;
  Range rg("hprqp_iterate");
  if (h->prm.launch_mode == 2) return solve_stream(h, t0, t1, lamA, lamQ, sigma);
  if (h->prm.launch_mode == 3) return solve_persist(h, t0, t1, lamA, lamQ, sigma);
  bool time_up = false;
  // ---- Algorithm 4 in launches of the fixed-schedule graph while fixed_L steps remain
  build_fixed(h);
  int64_t k0 = 0;
  if (h->g_fixed && max_iter >= h->fixed_L) {
    for (; max_iter - k0 >= h->fixed_L; k0 += h->fixed_L) {
      CU(h, cudaGraphLaunch(h->g_fixed, h->stream));
      h->launches += h->fixed_kernels;
      h->fixed_steps += h->fixed_L;
      CU(h, cudaMemcpyAsync(&h->hflags[0], &h->dctrl->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
      CU(h, cudaStreamSynchronize(h->stream));
      if (h->hflags[0]) return finish_solve(h, t0, t1, lamA, lamQ, sigma, false);
      if (h->prm.time_limit > 0 &&
          std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > h->prm.time_limit)
        return finish_solve(h, t0, t1, lamA, lamQ, sigma, true);
    }
    // a restart decided at the last fixed step runs before the dynamic graph's first step
    CU(h, launch_restart(a, h->plan, h->stream));
    h->launches += kernels_per_restart(a);
  }
  // ---- the rest in launches of the dynamic graph (iters_per_launch steps, built when first
  // needed); double-buffered done poll
  if ((st = build_iter_graph(h))) return st;
  const int64_t per = h->prm.iters_per_launch;
  const int64_t max_launch = (max_iter - k0 + per - 1) / per + 2;
  const int64_t nodes = h->conditional ? 1 : per * kernels_per_iteration(a);
  for (int64_t i = 0; i < max_launch; i++) {
    CU(h, cudaGraphLaunch(h->g_iter, h->stream));
    h->launches += nodes;
    CU(h, cudaMemcpyAsync(&h->hflags[i & 1], &h->dctrl->done, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaEventRecord(h->ev[i & 1], h->stream));
    if (i > 0) {
      CU(h, cudaEventSynchronize(h->ev[(i - 1) & 1]));
      if (h->hflags[(i - 1) & 1]) break;
    }
    if (h->prm.time_limit > 0) {
      double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (el > h->prm.time_limit) {
        time_up = true;
        break;
      }
    }
  }
  return finish_solve(h, t0, t1, lamA, lamQ, sigma, time_up);
}

static hprqp_status finish_solve(hprqp_handle* h, std::chrono::steady_clock::time_point t0,
                                 std::chrono::steady_clock::time_point t1, double lamA, double lamQ, double sigma,
                                 bool time_up) {
  Args& a = h->args;
  Ctrl& C = *h->hctrl;
  CU(h, cudaMemcpyAsync(h->hctrl, h->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  auto t2 = std::chrono::steady_clock::now();
  int status = C.status;
  if (!C.done) status = time_up ? HPRQP_TIME_LIMIT : HPRQP_MAX_ITER;
  hprqp_kkt& K = h->kkt;
  std::memset(&K, 0, sizeof(K));
  K.lanes_q = h->plan.gQ;
  K.lanes_a = h->plan.gA;
  K.lanes_at = h->plan.gAT;
  K.lanes_pre = h->plan.gPre;
  for (int f = 0; f < h->args.Q.nfac; f++) K.tiled_terms += h->args.Q.tiled[f];
  K.eta_p = C.eta_p;
  K.eta_d = C.eta_d;
  K.eta_gap = C.eta_gap;
  K.rel_kkt = std::max(C.eta_p, std::max(C.eta_d, C.eta_gap));
  K.pobj = C.pobj;
  K.dobj = C.dobj;
  K.iters = C.k;
  K.restarts = C.r;
  K.sigma = C.sigma;
  K.lambda_A = lamA;
  K.lambda_Q = lamQ;
  K.solve_seconds = std::chrono::duration<double>(t2 - t0).count();
  K.power_seconds = std::chrono::duration<double>(t1 - t0).count();
  // conditional graph and stream launches: only the variants taken ran kernels (the fixed graph's
  // launches were counted as launched, restarts apart)
  if (h->conditional || h->prm.launch_mode == 2)
    h->launches += std::max<int64_t>(0, C.k - h->fixed_steps) * kernels_per_step(a) + C.r * kernels_per_restart(a);
  K.kernel_launches = h->launches;
  K.status = status;
  // tolerance ladder: iterations and time (power method + device time since the first step)
  const int64_t lk[2] = {C.ladder_k[0], C.ladder_k[1]};
  for (int q = 0; q < 2; q++) {
    const double sec = lk[q] > 0 ? K.power_seconds + 1e-9 * (double)(C.ladder_ns[q] - C.t0_ns) : 0.0;
    if (q == 0) {
      K.iters_1e4 = lk[0];
      K.seconds_1e4 = sec;
    } else {
      K.iters_1e6 = lk[1];
      K.seconds_1e6 = sec;
    }
  }
  h->last_status = status;
  h->solved = true;
  h->last_lamA = lamA;
  h->last_lamQ = lamQ;
  h->last_sigma0 = sigma;
  return (hprqp_status)status;
}

extern "C" hprqp_status hprqp_history(hprqp_handle* h, hprqp_check* out, int32_t cap, int32_t* count) {
  if (!h || !count || cap < 0 || (cap > 0 && !out)) return HPRQP_INVALID_ARG;
  if (!h->solved) return fail(h, HPRQP_INVALID_ARG, "hprqp_history before hprqp_solve");
  static_assert(sizeof(hprqp_check) == sizeof(CheckRec), "record layouts differ");
  const long long total = h->prm.method != 0 ? 0 : h->hctrl->hist_n;
  const int64_t kept = std::min<long long>(total, kHistCap);
  const int64_t nout = std::min<int64_t>(kept, cap);
  std::vector<CheckRec> ring(kHistCap);
  CU(h, cudaMemcpy(ring.data(), h->args.hist, sizeof(CheckRec) * kHistCap, cudaMemcpyDeviceToHost));
  // the last nout records, oldest first
  for (int64_t i = 0; i < nout; i++) {
    const long long idx = (total - nout + i) % kHistCap;
    std::memcpy(&out[i], &ring[idx], sizeof(CheckRec));
  }
  *count = (int32_t)nout;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_profile(hprqp_handle* h, int32_t iters, double* ms) {
  if (!h) return HPRQP_INVALID_ARG;
  if (!h->solved) return fail(h, HPRQP_INVALID_ARG, "hprqp_profile before hprqp_solve");
  if (iters < 1 || !ms) return fail(h, HPRQP_INVALID_ARG, "need iters >= 1 and an output array");
  Range rg("hprqp_profile");
  hprqp_status st;
  if ((st = init_state(h, h->last_lamA, h->last_lamQ, h->last_sigma0, 1e-300, (int64_t)iters + 1))) return st;
  cudaEvent_t ev[HPRQP_PROF_KINDS][2];
  for (auto& e : ev) {
    CU(h, cudaEventCreate(&e[0]));
    CU(h, cudaEventCreate(&e[1]));
  }
  double tot[HPRQP_PROF_KINDS] = {0};
  int cnt[HPRQP_PROF_KINDS] = {0};
  double tot_all[HPRQP_PROF_KINDS] = {0};
  int cnt_all[HPRQP_PROF_KINDS] = {0};
  cudaError_t err = cudaSuccess;
  Ctrl& C = *h->hctrl;
  bool k1 = true;   // false: the previous step's fused pass ran this step's k_zx
  for (int32_t i = 0; i < iters && err == cudaSuccess; i++) {
    // the variant the device controller would select for this step
    const int var = C.done ? 3 : C.ttest ? 2 : C.rtest ? 1 : 0;
    if (var == 3) break;
    for (auto& e : ev) {  // fresh events: kinds a step does not launch stay unrecorded
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
      cudaEventCreate(&e[0]);
      cudaEventCreate(&e[1]);
    }
    // as in the fixed-schedule graph: a plain step that is not the last one profiled ends with
    // the fused passes, for the variant the controller will give the next step (no restart can
    // follow a plain step: k and t advance by one)
    int fuse_next = -1;
    if (h->plan.fuse && var == 0 && i + 1 < iters) {
      const long long k2 = C.k + 2;
      const bool nr = !C.restart_off && k2 % C.restart_every == 0;
      const bool nt = k2 % C.check_every == 0 || k2 >= C.max_iter;
      fuse_next = nt ? 2 : nr ? 1 : 0;
    }
    err = launch_step_fused(h->args, h->plan, h->stream, var, k1, fuse_next, ev);
    k1 = fuse_next < 0;
    if (err == cudaSuccess) err = cudaMemcpyAsync(h->hctrl, h->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (err == cudaSuccess && C.restart_pending && !C.done) {
      err = launch_restart(h->args, h->plan, h->stream, ev);
      if (err == cudaSuccess) err = cudaMemcpyAsync(h->hctrl, h->dctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, h->stream);
      if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    }
    for (int k = 0; k < HPRQP_PROF_KINDS && err == cudaSuccess; k++) {
      float t = 0.f;
      if (cudaEventElapsedTime(&t, ev[k][0], ev[k][1]) == cudaSuccess) {
        // step kernels: plain steps (the R~ and stopping-test variants carry extra sums);
        // every step's times are kept for a run without a plain step
        const bool plain_kind = k < HPRQP_PROF_RPRE || k >= HPRQP_PROF_ATH;
        if (!plain_kind || var == 0) {
          tot[k] += t;
          cnt[k]++;
        }
        tot_all[k] += t;
        cnt_all[k]++;
      } else {
        cudaGetLastError();
      }
    }
  }
  for (auto& e : ev) {
    cudaEventDestroy(e[0]);
    cudaEventDestroy(e[1]);
  }
  if (err != cudaSuccess) return fail(h, HPRQP_CUDA_ERROR, "profile: %s", cudaGetErrorString(err));
  for (int k = 0; k < HPRQP_PROF_KINDS; k++)
    ms[k] = cnt[k] ? tot[k] / cnt[k] : cnt_all[k] ? tot_all[k] / cnt_all[k] : 0.0;
  h->solved = false;  // the iterate no longer belongs to a solve
  return HPRQP_OK;
}

// ------------------------------------------------------------------------------------ get / apply
static hprqp_status copy_out(hprqp_handle* h, double* dst, const double* src, size_t count) {
  if (!dst || count == 0) return HPRQP_OK;
  CU(h, cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, h->stream));
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_get(hprqp_handle* h, double* x, double* y, double* z, double* w, hprqp_kkt* kkt) {
  if (!h) return HPRQP_INVALID_ARG;
  if (!h->solved) return fail(h, HPRQP_INVALID_ARG, "hprqp_get before hprqp_solve");
  Range rg("hprqp_get");
  hprqp_status st;
  Vec& V = h->args.V;
  if (z && h->last_status == HPRQP_TIME_LIMIT) CU(h, launch_zbar(h->args, h->plan, h->stream));
  const double *xs = V.xb, *ys = V.yb, *zs = V.zb, *ws = V.wb;
  if (h->scaled) {
    // back to the original variables: x = D xs, y = E ys, z = D^{-1} zs, w = D ws
    CU(h, launch_vmul_to(h->ux, V.xb, V.sd, h->n, h->stream));
    CU(h, launch_vmul_to(h->uy, V.yb, V.se, h->m, h->stream));
    CU(h, launch_vmul_to(h->uz, V.zb, V.isd, h->n, h->stream));
    CU(h, launch_vmul_to(h->uw, V.wb, V.sd, h->n, h->stream));
    xs = h->ux;
    ys = h->uy;
    zs = h->uz;
    ws = h->uw;
  }
  if ((st = copy_out(h, x, xs, h->n))) return st;
  if ((st = copy_out(h, y, ys, h->m))) return st;
  if ((st = copy_out(h, z, zs, h->n))) return st;
  if ((st = copy_out(h, w, ws, h->n))) return st;
  CU(h, cudaStreamSynchronize(h->stream));
  if (kkt) *kkt = h->kkt;
  return HPRQP_OK;
}

extern "C" hprqp_status hprqp_apply(hprqp_handle* h, int32_t op, const double* in, double* out) {
  if (!h) return HPRQP_INVALID_ARG;
  if (op < 0 || op > 2 || !in || !out) return fail(h, HPRQP_INVALID_ARG, "bad apply arguments");
  if (op <= 1 && h->m == 0) return fail(h, HPRQP_INVALID_ARG, "problem has no A rows");
  const int64_t nin = op == 0 ? h->n : op == 1 ? h->m : h->n;
  const int64_t nout = op == 0 ? h->m : h->n;
  Vec& V = h->args.V;
  CU(h, cudaMemcpyAsync((void*)V.ain, in, nin * sizeof(double), cudaMemcpyDefault, h->stream));
  // with preconditioning the stored operators are E A D, D A^T E, D Q D: map the input into
  // the scaled variables and the output back (A x = E^{-1} A_s D^{-1} x, and so on)
  if (h->scaled) CU(h, launch_vmul((double*)V.ain, op == 1 ? V.ise : V.isd, nin, h->stream));
  CU(h, launch_apply(h->args, h->plan, op, h->stream));
  if (h->scaled) CU(h, launch_vmul(V.aout, op == 0 ? V.ise : V.isd, nout, h->stream));
  CU(h, cudaMemcpyAsync(out, V.aout, nout * sizeof(double), cudaMemcpyDefault, h->stream));
  CU(h, cudaStreamSynchronize(h->stream));
  return HPRQP_OK;
}
