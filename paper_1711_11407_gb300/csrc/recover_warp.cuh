// The register-FFT recovery kernel k_recover_w (one warp per line, L in {32, 64, 128, 256}).
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
#pragma once

#include "recover_common.cuh"

// ---- warp-per-line variant for L = 32 R (R = 1, 2, 4, 8) ----------------------------------------
// One CTA of D+1 warps per signal; warp j gathers line j straight into registers and transforms it
// with warp_fft (no shared-memory staging, no CTA barrier inside the FFT).  Shared memory holds
// only the bins (bank-swizzled), the twiddles and the bucket set, so several times more signals
// are resident per SM than with the shared-memory Stockham path.
struct WLayout {
  size_t bins, tw, head, la, lk, nxt, stg, total;
};

static __host__ __device__ WLayout recover_layout_w(int D, int L_max, int k_cap, bool staged = false) {
  auto al = [](size_t v) -> size_t { return (v + 15) & ~size_t(15); };
  size_t P = 1;
  while (P < (size_t)k_cap) P <<= 1;
  const size_t lines = (size_t)(D + 1) * L_max * sizeof(float2);
  const size_t sortb = 2 * P * sizeof(int);
  WLayout w{};
  size_t off = 0;
  w.bins = off; off = al(off + (lines > sortb ? lines : sortb));
  w.tw = off; off = al(off + (size_t)L_max * sizeof(float2));
  w.head = off; off = al(off + (size_t)L_max * sizeof(int));
  w.la = off; off = al(off + (size_t)k_cap * sizeof(float2));
  w.lk = off; off = al(off + (size_t)D * k_cap * sizeof(int));
  w.nxt = off; off = al(off + (size_t)k_cap * sizeof(int));
  w.stg = off; off = al(off + (staged ? lines : 0));
  w.total = off;
  return w;
}

template <int D, int R>
__device__ __forceinline__ void fft_store_w(float2 (&v)[R], float2* bins, const Shape& sh, const float2* tw, int j,
                                            int lane, float invL) {
  warp_fft<R>(v, tw, sh.L, lane);
  const int br = brev5(lane);
  float2* out = bins + j * sh.L;
#pragma unroll
  for (int k2 = 0; k2 < R; ++k2) out[swz(k2 + R * br)] = cscale(v[k2], invL);
}

// Sanitised slope and offset of schedule row t (every entry reduced into [0, N_d)).
template <int D>
__device__ __forceinline__ void sched_row(const Shape& sh, const int* al, const int* ta, int* alr, int* tar) {
#pragma unroll
  for (int d = 0; d < D; ++d) {
    alr[d] = fmod_(__ldg(al + d) & 0x3fffffff, sh.fdims[d]);
    tar[d] = fmod_(__ldg(ta + d) & 0x3fffffff, sh.fdims[d]);
  }
}

// A schedule row as read from memory, loaded an iteration before its gather so that the sample
// addresses do not wait for the row (the L2-hint mode's pipeline).
template <int D>
struct RawRow {
  int a[D], t[D];
  __device__ __forceinline__ void load(const int* al, const int* ta) {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      a[d] = __ldg(al + d);
      t[d] = __ldg(ta + d);
    }
  }
  __device__ __forceinline__ void sanitize(const Shape& sh, int* alr, int* tar) const {
#pragma unroll
    for (int d = 0; d < D; ++d) {
      alr[d] = fmod_(a[d] & 0x3fffffff, sh.fdims[d]);
      tar[d] = fmod_(t[d] & 0x3fffffff, sh.fdims[d]);
    }
  }
};

template <int D>
__device__ __forceinline__ void peel_set_w(float2* bins, const Shape& sh, const BucketSet& s, int count, const int* ca,
                                           const int* ct, const float2* __restrict__ tw) {
  const int L = sh.L;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    int k[D];
    int msum = 0, psum = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      k[d] = s.lk[d * s.k_cap + i];
      msum += ca[d] * k[d];
      psum += ct[d] * k[d];
    }
    const int m = fmod_(msum, sh.fL);
    const int p = fmod_(psum, sh.fL);
    s.nxt[i] = atomicExch(&s.head[m], i);
    const float2 a = s.la[i];
    const int pm = swz(m);
    float2 v = cmulc(a, tw[p]);
    atomicAdd(&bins[pm].x, -v.x);
    atomicAdd(&bins[pm].y, -v.y);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      int q = p + sh.c[d] * k[d];
      if (q >= L) q -= L;
      v = cmulc(a, tw[q]);
      atomicAdd(&bins[(d + 1) * L + pm].x, -v.x);
      atomicAdd(&bins[(d + 1) * L + pm].y, -v.y);
    }
  }
}

template <int D>
__device__ __forceinline__ void decode_bins_w(const float2* bins, const Shape& sh, const BucketSet& s, const int* ca,
                                              const int* ct, const float2* __restrict__ tw, const Thresholds& th,
                                              int* t0, int* ovf, int* accepted) {
  const int L = sh.L;
  int my_t0 = 0, my_acc = 0;
  bool my_ovf = false;
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    const int pm = swz(m);
    const float2 s0 = bins[pm];
    float2 sd[D];
#pragma unroll
    for (int d = 0; d < D; ++d) sd[d] = bins[(d + 1) * L + pm];
    int k[D];
    bool counted = false;
    int v = th.fp64_all ? kUndecided : classify_fp32<D>(s0, sd, sh, th, k, &counted);
    if (v == kUndecided) {
      bool c64 = false;
      v = classify_fp64<D>(s0, sd, sh, th, k, &c64);
      counted = c64;
    }
    my_t0 += counted ? 1 : 0;
    if (v != kAccept) continue;
    int msum = 0, psum = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      msum += ca[d] * k[d];
      psum += ct[d] * k[d];
    }
    if (fmod_(msum, sh.fL) != m) continue;                            // T3
    const float2 a = decoded_amplitude<D>(s0, sd, sh, k, fmod_(psum, sh.fL), tw, th.amp_average != 0);
    ++my_acc;
    if (!bucket_insert<D>(s, m, k, a)) my_ovf = true;
  }
  if (my_t0) atomicAdd(t0, my_t0);
  if (my_acc) atomicAdd(accepted, my_acc);
  if (my_ovf) atomicOr(ovf, 1);
}

// When every bin that passed T0 in iteration t-1 was decoded and merged, the set is most likely
// complete and iteration t will find nothing (the early stop): iteration t then does not prefetch
// t+1.  If the guess is wrong, iteration t+1 gathers its samples synchronously; the results do not
// depend on the guess.
// WM: how iteration t+1's samples are requested during iteration t.  kWPrefetch: into registers
// right after the FFT; kWStaged: into shared memory by cp.async; kWNone: not at all (iteration t+1
// gathers synchronously; with many signals per SM the other CTAs hide that latency, and the
// registers the prefetch would hold are freed); kWL2Hint: as kWNone, but the samples are hinted
// into L2 right after the FFT and the schedule rows are read an iteration ahead (few signals per
// SM: the synchronous gather then waits for L2, not DRAM).  A CTA barrier waits for the loads its
// threads have outstanding, so register prefetches only overlap the work before the next barrier.
constexpr int kWPrefetch = 0, kWStaged = 1, kWNone = 2, kWL2Hint = 3;

template <int D, int R, int WM>
__device__ __forceinline__ int iterate_w(const RecoverArgs& A, const Shape& sh, const BucketSet& set, float2* bins,
                                         const float2* tws, float2* stg, const float2* __restrict__ x,
                                         const int* sched_a, const int* sched_t, int T, int warp, int lane,
                                         float invL, int* s_ca, int* s_ct, int* s_t0, int* s_ovf, int* s_acc) {
  constexpr bool STAGED = WM == kWStaged;
  const int L = sh.L;
  float2 nxt[WM == kWPrefetch ? R : 1];
  float2* my_stg = stg + warp * L;
  bool have_next = false;      // samples of the current iteration already requested
  bool likely_done = false;    // every T0 bin of the previous iteration was accepted
  constexpr bool HINT = WM == kWL2Hint;
  constexpr bool SYNC = WM == kWNone || WM == kWL2Hint;   // every iteration gathers at its start
  FPSSFT_PH(kPhSetup);
  RawRow<D> cur, nx;   // kWL2Hint: schedule rows t and t+1
  if (HINT) {
    if (T > 0) cur.load(sched_a, sched_t);
    if (T > 1) nx.load(sched_a + D, sched_t + D);
  }
  if (T > 0 && !SYNC) {   // without prefetch the first iteration gathers like every other
    int alr[D], tar[D];
    sched_row<D>(sh, sched_a, sched_t, alr, tar);
    if (STAGED)
      gather_line_async<D, R>(my_stg, x, sh, alr, tar, warp, lane);
    else
      gather_line_regs<D, (WM == kWPrefetch ? R : 1)>(nxt, x, sh, alr, tar, warp, lane);
    have_next = true;
  }
  int iters = 0;
  for (int t = 0; t < T; ++t) {
    const int* al = sched_a + t * D;
    const int* ta = sched_t + t * D;
    if (threadIdx.x < D) {
      const int d = threadIdx.x;
      s_ca[d] = cmodL(sh, d, HINT ? cur.a[d] : al[d]);
      s_ct[d] = cmodL(sh, d, HINT ? cur.t[d] : ta[d]);
    }
    for (int m = threadIdx.x; m < L; m += blockDim.x) set.head[m] = -1;
    float2 v[R];
    if (!have_next) {
      int alr[D], tar[D];
      if (HINT)
        cur.sanitize(sh, alr, tar);
      else
        sched_row<D>(sh, al, ta, alr, tar);
      gather_line_regs<D, R>(v, x, sh, alr, tar, warp, lane);
    } else if (STAGED) {
      cp_async_wait<0>();
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = my_stg[lane + 32 * i];
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = nxt[WM == kWPrefetch ? i : 0];
    }
    FPSSFT_PH(kPhGather);
    fft_store_w<D, R>(v, bins, sh, tws, warp, lane, invL);    // consumes v: the reads above are done
    FPSSFT_PH(kPhFft);
    have_next = !SYNC && t + 1 < T && !likely_done;
    if (have_next) {
      int alr[D], tar[D];
      sched_row<D>(sh, al + D, ta + D, alr, tar);
      if (STAGED)
        gather_line_async<D, R>(my_stg, x, sh, alr, tar, warp, lane);
      else
        gather_line_regs<D, (WM == kWPrefetch ? R : 1)>(nxt, x, sh, alr, tar, warp, lane);
    }
    if (HINT) {
      if (t + 1 < T) {
        int alr[D], tar[D];
        nx.sanitize(sh, alr, tar);
        prefetch_line_l2<D, R>(x, sh, alr, tar, warp, lane);
      }
      cur = nx;                                                // row t is no longer needed
      if (t + 2 < T) nx.load(sched_a + (t + 2) * D, sched_t + (t + 2) * D);
    }
    __syncthreads();
    FPSSFT_PH(kPhGather);
    if (threadIdx.x == 0) {
      *s_t0 = 0;
      *s_acc = 0;
    }
    peel_set_w<D>(bins, sh, set, min(*set.count, A.k_cap), s_ca, s_ct, tws);
    __syncthreads();
    FPSSFT_PH(kPhPeel);
    decode_bins_w<D>(bins, sh, set, s_ca, s_ct, tws, A.th, s_t0, s_ovf, s_acc);
    __syncthreads();
    FPSSFT_PH(kPhDecode);
    iters = t + 1;
    const bool stop = (A.early_stop && *s_t0 == 0) || *s_ovf != 0 || (A.early_stop == 2 && *s_acc == *s_t0);
    if (stop) break;
    likely_done = A.early_stop && *s_acc == *s_t0;
  }
  if (STAGED) cp_async_wait<0>();   // a copy issued past the last iteration lands before reuse
  return iters;
}

#ifndef FPSSFT_W_THREADS_PER_SM
#define FPSSFT_W_THREADS_PER_SM 640   // resident threads per SM the warp path's register budget targets
#endif

#ifndef FPSSFT_WS_THREADS_PER_SM
// same for the variant that stages the prefetch in shared memory, the latency variant: a generous
// budget (no spills; 768 threads per SM spilled and ran 1.6x slower on 256 noisy 64^3 cubes)
#define FPSSFT_WS_THREADS_PER_SM 384
#endif

template <int D, int WM>
__global__ void __launch_bounds__(32 * (D + 1), (WM == kWStaged ? FPSSFT_WS_THREADS_PER_SM : FPSSFT_W_THREADS_PER_SM) / (32 * (D + 1)))
    k_recover_w(RecoverArgs A) {
  constexpr bool STAGED = WM == kWStaged;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_sig, s_count, s_t0, s_ovf, s_n, s_acc;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  __shared__ int s_cnt[kOutBuckets], s_off[kOutBuckets];
  const WLayout lay = recover_layout_w(D, A.L_max, A.k_cap, STAGED);
  float2* bins = reinterpret_cast<float2*>(smem + lay.bins);
  float2* tws = reinterpret_cast<float2*>(smem + lay.tw);
  float2* stg = reinterpret_cast<float2*>(smem + lay.stg);
  BucketSet set;
  set.lk = reinterpret_cast<int*>(smem + lay.lk);
  set.la = reinterpret_cast<float2*>(smem + lay.la);
  set.head = reinterpret_cast<int*>(smem + lay.head);
  set.nxt = reinterpret_cast<int*>(smem + lay.nxt);
  set.count = &s_count;
  set.k_cap = A.k_cap;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
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
      load_shape(sh, A.tab.shapes, si, tws, A.tab.twiddles, true);
      loaded = si;
    }
    if (threadIdx.x == 0) {
      s_count = 0;
      s_ovf = 0;
    }
    __syncthreads();
    const int L = sh.L;
    const int R = L >> 5;
    const float invL = 1.0f / (float)L;
    const float2* x = A.cubes + A.offsets[b];
    int* ok_out = A.out_k + (size_t)b * A.k_cap * D;
    float2* oa_out = A.out_a + (size_t)b * A.k_cap;

    if (A.init_count != nullptr) {   // resume: the caller's set is appended as given
      const int n0 = min(max(A.init_count[b], 0), A.k_cap);
      for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        int k[D];
#pragma unroll
        for (int d = 0; d < D; ++d) k[d] = ok_out[i * D + d];
        if (!on_grid<D>(sh, k)) continue;
        const int idx = atomicAdd(&s_count, 1);
#pragma unroll
        for (int d = 0; d < D; ++d) set.lk[d * A.k_cap + idx] = k[d];
        set.la[idx] = oa_out[i];
      }
      __syncthreads();
    }

    const int T = A.tab.sig_T[b];
    const int* sched_a = A.alpha + (size_t)b * A.sched_stride;
    const int* sched_t = A.tau + (size_t)b * A.sched_stride;
    int iters = 0;
    switch (R) {
      case 1: iters = iterate_w<D, 1, WM>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      case 2: iters = iterate_w<D, 2, WM>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      case 4: iters = iterate_w<D, 4, WM>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      default: iters = iterate_w<D, 8, WM>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
    }
    FPSSFT_PH_ITERS(iters);

    const int count = min(s_count, A.k_cap);
    int* tkey = reinterpret_cast<int*>(bins);                        // the bins are free now
    int* tidx = tkey + (lay.tw - lay.bins) / (2 * sizeof(int));
    auto key_of = [&](int i) {
      int key = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) key += set.lk[d * A.k_cap + i] * sh.strides[d];
      return key;
    };
    auto put = [&](int r, int i) {
#pragma unroll
      for (int d = 0; d < D; ++d) ok_out[r * D + d] = set.lk[d * A.k_cap + i];
      oa_out[r] = set.la[i];
    };
    auto amp_of = [&](int i) { return set.la[i]; };
    const int n = emit_bucketed(count, sh.N, A.th, tkey, tidx, s_cnt, s_off, &s_n, amp_of, key_of, put);
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
