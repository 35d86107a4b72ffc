// Persistent form of the single-instance solver: all passes of Algorithm 4 in one cooperative
// launch, separated by grid barriers instead of kernel boundaries.
//
// Small and mid-sized problems spend most of an inner step in launch latency and in the ramp
// and tail of seven short kernels.  Here every block of a co-resident grid runs the same pass
// bodies as the separate kernels (the run-time variants, which read the restart / stopping
// flags from the controller), waits at a grid barrier after each pass, and loops over inner
// steps until the controller marks the solve done or the launch's step budget is used up.
// The bodies are compiled with coherent loads (HPRQP_COHERENT): vectors written by other
// blocks earlier in the same launch are read through L2, never through the read-only cache.
//
// The grid barrier is a generation counter.  Every wait is bounded; a block whose wait gives
// up records an error flag and leaves its loop, so the others give up at their next barrier
// and the launch ends with the flag set (the host reports HPRQP_TIMEOUT).
#define HPRQP_COHERENT 1
#include "kernels.cuh"

namespace hprqp {
namespace {

constexpr unsigned kBarSpin = 1u << 24;   // default polls of one barrier wait (well over a second)

// bar[0]: arrivals, bar[1]: generation; err: set when a wait gives up after `spin` polls
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, unsigned spin) {
  __shared__ int ok;
  __syncthreads();
  if (gridDim.x == 1) return true;
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* gen_p = bar + 1;
    const unsigned gen = *gen_p;
    __threadfence();
    if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&bar[0], 0u);
      __threadfence();
      atomicAdd(&bar[1], 1u);
    } else {
      for (unsigned i = 0; *gen_p == gen; ++i) {
        if (i >= spin || *(volatile int*)err) {
          atomicExch(err, 1);
          ok = 0;
          break;
        }
        if (i >= 32) __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

#define HPRQP_ROWS(KIND, GSEL)                                      \
  do {                                                              \
    if ((GSEL) == 1) rows_body<1, KIND, VAR_RUNTIME>(a, none);       \
    else rows_body<4, KIND, VAR_RUNTIME>(a, none);                   \
  } while (0)

#define HPRQP_PRE(TT, WHICH)                        \
  do {                                              \
    if (p.gpre == 1) pre_body<1, TT>(a, WHICH);      \
    else pre_body<8, TT>(a, WHICH);                  \
  } while (0)

#define HPRQP_SYNC() \
  if (!grid_barrier(p.bar, p.err, p.spin)) return

struct PersistParams {
  int gq, ga, gat, gpre;   // lanes per row (1 or 4) and of the pre-pass (1 or 8)
  long long steps;         // inner steps of this launch at most
  unsigned* bar;
  int* err;
  unsigned spin;           // polls of one barrier wait before it gives up
};

__global__ void __launch_bounds__(kThreads) k_persist(Args a, PersistParams p) {
  const Handles none;
  Ctrl* C = a.C;
  const bool HQ = a.Q.present(), HA = a.m > 0, pre = a.Q.has_fd();   // (no QAP term here)
  for (long long it = 0; it < p.steps; ++it) {
    if (*(volatile int*)&C->done) return;
    // one inner step, in the order of the separate launches
    zx_body<VAR_RUNTIME>(a);
    HPRQP_SYNC();
    if (HQ) {
      if (pre) {
        HPRQP_PRE(2, 0);
        HPRQP_SYNC();
      }
      HPRQP_ROWS(K_Q1, p.gq);
      HPRQP_SYNC();
    }
    if (HA) {
      HPRQP_ROWS(K_A1, p.ga);
      HPRQP_SYNC();
      HPRQP_ROWS(K_AT, p.gat);
      HPRQP_SYNC();
      if (HQ) {
        if (pre) {
          HPRQP_PRE(0, 1);
          HPRQP_SYNC();
        }
        HPRQP_ROWS(K_Q2, p.gq);
        HPRQP_SYNC();
      }
    }
    if (!HQ && !HA) {
      HPRQP_ROWS(K_AT, p.gat);
      HPRQP_SYNC();
    }
    // restart pass (theta~ of eq. (3.11), Algorithm 5) when the controller asked for one
    if (*(volatile int*)&C->restart_pending && !*(volatile int*)&C->done) {
      if (HQ && HA && pre) {
        HPRQP_PRE(0, 2);
        HPRQP_SYNC();
      }
      if (p.gq == 1) restart_body<1>(a);
      else restart_body<4>(a);
      HPRQP_SYNC();
    }
  }
}

#undef HPRQP_ROWS
#undef HPRQP_PRE
#undef HPRQP_SYNC

// the persistent kernel carries two lane widths per pass (short and long rows)
int snap_rows(int g) { return g <= 2 ? 1 : 4; }
int snap_pre(int g) { return g <= 2 ? 1 : 8; }

}  // namespace

int persist_max_blocks(int sms) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_persist, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return occ * sms;
}

cudaError_t launch_persist(const Args& a, const Plan& pl, int grid, long long steps, unsigned* bar, int* err,
                           unsigned spin, cudaStream_t s) {
  Args ag = a;
  ag.nbM = grid;   // the y-step partials of this launch have one row per block
  PersistParams p;
  p.gq = snap_rows(pl.gQ);
  p.ga = snap_rows(pl.gA);
  p.gat = snap_rows(pl.gAT);
  p.gpre = snap_pre(pl.gPre);
  p.steps = steps;
  p.bar = bar;
  p.err = err;
  p.spin = spin > 0 ? spin : kBarSpin;
  void* args[] = {&ag, &p};
  return cudaLaunchCooperativeKernel((const void*)k_persist, dim3(grid), dim3(kThreads), args, 0, s);
}

}  // namespace hprqp
