// Optional per-phase cycle counters of the recovery kernels (tracing).
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by
// recover_common.cuh.
//
// Compiled in only with -DFPSSFT_PHASE_TIMERS; otherwise every macro below expands to nothing and
// the kernels are the same as without this file.  With it, thread 0 of each CTA keeps in shared
// memory the SM clock cycles (clock64) spent in each phase of the recovery loop.  Every mark is a
// CTA barrier first, so a phase ends when its slowest thread does; the extra barriers make the
// launch slower than the plain one.  At the end of the kernel each CTA adds to g_phase its
// counters, the iterations it ran, its total cycles and the global-timer nanoseconds of the same
// span (their ratio converts cycles to time at the clock the launch actually ran at);
// fpssft_phase_read copies g_phase out and clears it.  In the register path the wait for samples
// prefetched into registers falls where they are first read: the copy into the FFT's inputs (the
// gather phase), or the FFT itself where the compiler folds that copy away.
#pragma once

// Phase indices; the order is the one of FPSSFT_PHASE_COUNT's documentation in fpssft.h.
enum PhaseId { kPhSetup = 0, kPhGather, kPhFft, kPhPeel, kPhDecode, kPhExchange, kPhOutput, kNumPhases };
// g_phase: [0, kNumPhases) cycles per phase summed over CTAs, then CTAs, iterations, total cycles,
// total nanoseconds.
constexpr int kPhaseWords = kNumPhases + 4;

#ifdef FPSSFT_PHASE_TIMERS
__device__ unsigned long long g_phase[kPhaseWords];
__shared__ long long ph_acc[kNumPhases];
__shared__ long long ph_prev, ph_c0, ph_t0, ph_iters;

__device__ __forceinline__ long long ph_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

__device__ __forceinline__ void ph_start() {
  if (threadIdx.x == 0) {
    for (int i = 0; i < kNumPhases; ++i) ph_acc[i] = 0;
    ph_iters = 0;
    ph_t0 = ph_globaltimer();
    ph_c0 = ph_prev = clock64();
  }
  __syncthreads();
}

// Every thread of the CTA must reach each mark (it is a barrier).
__device__ __forceinline__ void ph_mark(int p) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long c = clock64();
    ph_acc[p] += c - ph_prev;
    ph_prev = c;
  }
}

__device__ __forceinline__ void ph_add_iters(int n) {
  if (threadIdx.x == 0) ph_iters += n;
}

__device__ __forceinline__ void ph_flush() {
  __syncthreads();
  if (threadIdx.x == 0) {
    const long long c = clock64();
    const long long t = ph_globaltimer();
    for (int i = 0; i < kNumPhases; ++i) atomicAdd(&g_phase[i], (unsigned long long)ph_acc[i]);
    atomicAdd(&g_phase[kNumPhases], 1ull);
    atomicAdd(&g_phase[kNumPhases + 1], (unsigned long long)ph_iters);
    atomicAdd(&g_phase[kNumPhases + 2], (unsigned long long)(c - ph_c0));
    atomicAdd(&g_phase[kNumPhases + 3], (unsigned long long)(t - ph_t0));
  }
}

#define FPSSFT_PH_START() ph_start()
#define FPSSFT_PH(p) ph_mark(p)
#define FPSSFT_PH_ITERS(n) ph_add_iters(n)
#define FPSSFT_PH_FLUSH() ph_flush()
#else
#define FPSSFT_PH_START() ((void)0)
#define FPSSFT_PH(p) ((void)0)
#define FPSSFT_PH_ITERS(n) ((void)0)
#define FPSSFT_PH_FLUSH() ((void)0)
#endif
