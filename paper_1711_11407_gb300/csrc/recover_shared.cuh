// The one-CTA-per-signal recovery kernel k_recover (shared-memory Stockham FFT, any L) and its
// global-workspace variant.
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
#pragma once

#include "recover_common.cuh"

// GM = true: the same kernel with the lines, the FFT partner and the recovered set in a per-CTA
// slice of global workspace (L2-resident) instead of shared memory, for lines or sets too large
// for one CTA's shared memory.  All device functions take generic pointers.
// Register budget: the 512-thread instance for D <= 2 keeps 64 registers so that two CTAs share an
// SM when shared memory allows (mid-length lines in large batches); for D >= 3 the longer decode
// needs more registers (at 64 it spills: the 64^3 batch ran twice as long).
template <int D, int MAXT, bool GM = false>
__global__ void __launch_bounds__(MAXT, (MAXT == 512 && D <= 2) ? 2 : 1) k_recover(RecoverArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_sig, s_count, s_t0, s_ovf, s_n, s_acc;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  __shared__ int s_cnt[kOutBuckets], s_off[kOutBuckets];

  unsigned char* base = GM ? A.gm_ws + (size_t)blockIdx.x * A.gm_stride : smem;
  const SmemLayout lay = recover_layout(D, A.L_max, A.k_cap, 1 << A.hash_bits, A.tw_smem != 0, A.prefetch != 0);
  float2* bufA = reinterpret_cast<float2*>(base + lay.bufA);
  float2* bufB = reinterpret_cast<float2*>(base + lay.bufB);
  float2* bufC = reinterpret_cast<float2*>(base + lay.bufC);
  const bool pf = A.prefetch != 0;
  float2* tws = reinterpret_cast<float2*>(base + lay.tw);
  float2* stws = reinterpret_cast<float2*>(base + lay.stw);
  SetView set;
  set.la = reinterpret_cast<float2*>(base + lay.la);
  set.lk = reinterpret_cast<int*>(base + lay.lk);
  set.lkey = reinterpret_cast<int*>(base + lay.lkey);
  set.hkey = reinterpret_cast<int*>(base + lay.hkey);
  set.hidx = reinterpret_cast<int*>(base + lay.hidx);
  set.count = &s_count;
  set.k_cap = A.k_cap;
  set.hash_bits = A.hash_bits;
  const int hash_cap = 1 << A.hash_bits;
  FPSSFT_PH_START();

  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) s_sig = claim_signal(A);
    __syncthreads();
    const int qi = s_sig;
    if (qi >= A.batch) break;
    const int b = A.tab.order[qi];
    const int si = A.tab.sig_shape[b];
    if (si != loaded) {
      load_shape(sh, A.tab.shapes, si, tws, A.tab.twiddles, A.tw_smem != 0);
      const int so = A.tab.shapes[si].stw_off;
      if (A.tw_smem && so >= 0) {
        const int L = A.tab.shapes[si].L;
        for (int i = threadIdx.x; i < L - 1; i += blockDim.x) stws[i] = A.tab.twiddles[so + i];
      }
      loaded = si;
    }
    for (int i = threadIdx.x; i < hash_cap; i += blockDim.x) set.hkey[i] = kEmpty;
    if (threadIdx.x == 0) {
      s_count = 0;
      s_ovf = 0;
    }
    __syncthreads();
    const float2* tw = A.tw_smem ? tws : A.tab.twiddles + sh.tw_off;
    const float2* stw = sh.stw_off < 0 ? nullptr : (A.tw_smem ? stws : A.tab.twiddles + sh.stw_off);
    const int L = sh.L;
    const float2* x = A.cubes + A.offsets[b];
    int* ok_out = A.out_k + (size_t)b * A.k_cap * D;
    float2* oa_out = A.out_a + (size_t)b * A.k_cap;

    if (A.init_count != nullptr) {   // resume from a given set
      const int n0 = min(max(A.init_count[b], 0), A.k_cap);
      for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        int k[D];
        int key = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          k[d] = ok_out[i * D + d];
          key += k[d] * sh.strides[d];
        }
        if (on_grid<D>(sh, k) && !set_insert<D>(set, k, key, oa_out[i])) atomicOr(&s_ovf, 1);
      }
      __syncthreads();
    }

    const int T = A.tab.sig_T[b];
    const int* sched_a = A.alpha + (size_t)b * A.sched_stride;
    const int* sched_t = A.tau + (size_t)b * A.sched_stride;
    FPSSFT_PH(kPhSetup);
    if (pf && T > 0) gather_lines_async<D>(bufA, x, sh, sched_a, sched_t);
    int iters = 0;
    for (int t = 0; t < T; ++t) {
      const int* al = sched_a + t * D;
      const int* ta = sched_t + t * D;
      if (threadIdx.x < D) {
        const int d = threadIdx.x;
        s_ca[d] = cmodL(sh, d, al[d]);
        s_ct[d] = cmodL(sh, d, ta[d]);
      }
      float2* cur = (pf && (t & 1)) ? bufC : bufA;
      if (pf) {
        // samples of t were requested one iteration ago; request t+1's now, wait for t's
        if (t + 1 < T) {
          gather_lines_async<D>((t & 1) ? bufA : bufC, x, sh, al + D, ta + D);
          cp_async_wait<1>();
        } else {
          cp_async_wait<0>();
        }
      } else if (A.gather_mode == 2) {
        gather_lines<D, 1>(bufA, x, sh, al, ta);
      } else {
        gather_lines<D, 0>(bufA, x, sh, al, ta);
      }
      __syncthreads();
      FPSSFT_PH(kPhGather);
      if (threadIdx.x == 0) {
        s_t0 = 0;
        s_acc = 0;
      }
      float2* bins = fft_lines(cur, bufB, D + 1, sh, tw, 1.0f / (float)L, stw);
      FPSSFT_PH(kPhFft);
      peel_set<D>(bins, sh, set, min(s_count, A.k_cap), s_ca, s_ct, tw);
      __syncthreads();
      FPSSFT_PH(kPhPeel);
      decode_bins<D>(bins, L, sh, set, s_ca, s_ct, tw, A.th, &s_t0, &s_ovf, &s_acc);
      __syncthreads();
      FPSSFT_PH(kPhDecode);
      iters = t + 1;
      const bool stop = (A.early_stop && s_t0 == 0) || s_ovf != 0 || (A.early_stop == 2 && s_acc == s_t0);
      if (stop) break;
    }

    if (pf) cp_async_wait<0>();   // a prefetch past the last iteration still lands before reuse
    FPSSFT_PH_ITERS(iters);
    // output: keep |a| > theta0, in order of linear index (hash arrays reused as sort buffers)
    const int count = min(s_count, A.k_cap);
    auto key_of = [&](int i) { return set.lkey[i]; };
    auto put = [&](int r, int i) {
#pragma unroll
      for (int d = 0; d < D; ++d) ok_out[r * D + d] = set.lk[d * A.k_cap + i];
      oa_out[r] = set.la[i];
    };
    auto amp_of = [&](int i) { return set.la[i]; };
    const int n = emit_bucketed(count, sh.N, A.th, set.hkey, set.hidx, s_cnt, s_off, &s_n, amp_of, key_of, put);
    if (threadIdx.x == 0) {
      A.out_count[b] = n;
      A.out_iters[b] = iters;
      A.out_status[b] = s_ovf ? kStatusCapacity : 0;
    }
    __syncthreads();
    FPSSFT_PH(kPhOutput);
  }
  FPSSFT_PH_FLUSH();
}
