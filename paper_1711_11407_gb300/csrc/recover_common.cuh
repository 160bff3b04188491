// Definitions shared by the recovery kernels and the host: the launch arguments, the shared-memory
// layout of the one-CTA-per-signal kernel and the per-signal shape loader.
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
#pragma once

#include <cuda_runtime.h>

#include "fpssft.h"
#include "fpssft_device.cuh"
#include "phase_timers.cuh"

using namespace fpssft;

constexpr int kStatusCapacity = FPSSFT_ERR_CAPACITY;

struct DeviceTables {
  const Shape* shapes;
  const int* sig_shape;
  const int* sig_T;
  const int* order;
  const float2* twiddles;
};

struct RecoverArgs {
  const float2* cubes;
  const int64_t* offsets;
  const int* alpha;
  const int* tau;
  int sched_stride;          // T_max * D
  DeviceTables tab;
  int* work_counter;         // 0 at launch; the launch's last claim returns it to 0 (claim_signal)
  int batch;
  int k_cap;
  int hash_bits;
  int L_max;
  int tw_smem;
  int prefetch;
  int gather_mode;
  int early_stop;
  unsigned char* gm_ws;      // lines and recovered set in global memory (lines longer than shared memory)
  size_t gm_stride;          // bytes of workspace per CTA
  Thresholds th;
  const int* init_count;
  int* out_k;
  float2* out_a;
  int* out_count;
  int* out_iters;
  int* out_status;
};

// Next queue position for a persistent recovery CTA (thread 0).  Every CTA claims until it draws a
// position past the batch, so a launch hands out exactly batch + gridDim.x positions; whoever draws
// the last one knows every claim of the launch has been made and returns the counter to 0, so the
// next launch on the stream needs no reset of its own.
__device__ __forceinline__ int claim_signal(const RecoverArgs& A) {
  const int c = atomicAdd(A.work_counter, 1);
  if (c == A.batch + (int)gridDim.x - 1) atomicExch(A.work_counter, 0);
  return c;
}

struct SmemLayout {
  size_t bufA, bufB, bufC, tw, stw, la, lk, lkey, hkey, hidx, total;
};

// bufA / bufC: the samples of iterations t and t+1 (bufC only when the gather is prefetched);
// bufB: the FFT's ping-pong partner.
static __host__ __device__ SmemLayout recover_layout(int D, int L_max, int k_cap, int hash_cap, bool tw_smem,
                                                     bool prefetch) {
  auto al = [](size_t v) -> size_t { return (v + 15) & ~size_t(15); };
  SmemLayout s{};
  size_t off = 0;
  const size_t lines = (size_t)(D + 1) * L_max * sizeof(float2);
  s.bufA = off; off = al(off + lines);
  s.bufB = off; off = al(off + lines);
  s.bufC = off; off = al(off + (prefetch ? lines : 0));
  s.tw = off; off = al(off + (tw_smem ? (size_t)L_max * sizeof(float2) : 0));
  s.stw = off; off = al(off + (tw_smem ? (size_t)L_max * sizeof(float2) : 0));   // per-stage twiddles
  s.la = off; off = al(off + (size_t)k_cap * sizeof(float2));
  s.lk = off; off = al(off + (size_t)D * k_cap * sizeof(int));
  s.lkey = off; off = al(off + (size_t)k_cap * sizeof(int));
  s.hkey = off; off = al(off + (size_t)hash_cap * sizeof(int));
  s.hidx = off; off = al(off + (size_t)hash_cap * sizeof(int));
  s.total = off;
  return s;
}

// Copy a Shape into shared memory (cooperatively) and, when twiddles live in shared memory, its
// twiddle table.  Caller synchronises afterwards.
__device__ __forceinline__ void load_shape(Shape& sh, const Shape* __restrict__ shapes, int si, float2* tws,
                                           const float2* __restrict__ twiddles, bool tw_smem) {
  const int* src = reinterpret_cast<const int*>(shapes + si);
  int* dst = reinterpret_cast<int*>(&sh);
  for (int i = threadIdx.x; i < (int)(sizeof(Shape) / sizeof(int)); i += blockDim.x) dst[i] = src[i];
  if (tw_smem) {
    const int L = shapes[si].L;
    const float2* t = twiddles + shapes[si].tw_off;
    for (int i = threadIdx.x; i < L; i += blockDim.x) tws[i] = t[i];
  }
}
