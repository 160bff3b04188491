// FPS-SFT recovery loop for GB300 (sm_103a): kernels and the C ABI declared in include/fpssft.h.
//
// Paper: Wang, Patel, Petropulu, "FPS-SFT: A Multi-dimensional Sparse Fourier Transform Based on
// the Fourier Projection-slice Theorem", arXiv 1711.11407.  The iteration of Sec. 2.2 (sample the
// D+1 lines, L-point DFT, subtract the recovered set, decode 1-sparse bins, merge) runs inside one
// launch for a whole batch, every signal owned by one CTA (or one cluster of CTAs) for all its
// iterations with its bins, twiddles and recovered set on chip, so the only global traffic per
// iteration is the (D+1) L sample gather.  Three kernels: k_recover_w (one warp per line, register
// FFT, for L in {32, 64, 128, 256}), k_recover (one persistent CTA per signal, shared-memory
// mixed-radix FFT, any L; with a global-workspace variant for lines or sets too large for shared
// memory) and k_recover_c (one CTA per line, the D+1 CTAs of a signal forming a thread-block cluster
// that exchanges bins through distributed shared memory; long lines in small batches).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "fpssft.h"
#include "fpssft_device.cuh"

using namespace fpssft;

namespace {

thread_local std::string g_last_error;

fpssft_status fail(fpssft_status st, const std::string& msg) {
  g_last_error = msg;
  return st;
}

#define FPSSFT_CUDA_TRY(call)                                                                    \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess) {                                                                     \
      return fail(FPSSFT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));         \
    }                                                                                            \
  } while (0)

constexpr int kStatusCapacity = FPSSFT_ERR_CAPACITY;

// The dynamic shared-memory limit is a property of the kernel (per device), shared by every plan:
// raise it when a plan needs more, never lower it under a plan that needs more.
// (fixed-size table: recording a limit allocates nothing)
struct AttrEntry {
  int dev;
  const void* func;
  int bytes;
};
std::mutex g_attr_mutex;
AttrEntry g_attr_tab[1024];
int g_attr_n = 0;

cudaError_t ensure_dynamic_smem(const void* func, size_t bytes) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(g_attr_mutex);
  AttrEntry* e = nullptr;
  for (int i = 0; i < g_attr_n && !e; ++i)
    if (g_attr_tab[i].dev == dev && g_attr_tab[i].func == func) e = &g_attr_tab[i];
  if (!e) {
    if (g_attr_n >= 1024) return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    e = &g_attr_tab[g_attr_n++];
    e->dev = dev;
    e->func = func;
    e->bytes = 0;
  }
  if ((int)bytes <= e->bytes) return cudaSuccess;
  const cudaError_t r = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (r == cudaSuccess) e->bytes = (int)bytes;
  return r;
}

struct DeviceTables {
  const Shape* shapes;
  const int* sig_shape;
  const int* sig_T;
  const int* order;
  const float2* twiddles;
};

}  // namespace

// ================================================================================================
// Kernels
// ================================================================================================

struct RecoverArgs {
  const float2* cubes;
  const int64_t* offsets;
  const int* alpha;
  const int* tau;
  int sched_stride;          // T_max * D
  DeviceTables tab;
  int* work_counter;
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

struct SmemLayout {
  size_t bufA, bufB, bufC, tw, la, lk, lkey, hkey, hidx, total;
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

// GM = true: the same kernel with the lines, the FFT partner and the recovered set in a per-CTA
// slice of global workspace (L2-resident) instead of shared memory, for lines or sets too large
// for one CTA's shared memory.  All device functions take generic pointers.
template <int D, int MAXT, bool GM = false>
__global__ void __launch_bounds__(MAXT) k_recover(RecoverArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_sig, s_count, s_t0, s_ovf, s_n;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];

  unsigned char* base = GM ? A.gm_ws + (size_t)blockIdx.x * A.gm_stride : smem;
  const SmemLayout lay = recover_layout(D, A.L_max, A.k_cap, 1 << A.hash_bits, A.tw_smem != 0, A.prefetch != 0);
  float2* bufA = reinterpret_cast<float2*>(base + lay.bufA);
  float2* bufB = reinterpret_cast<float2*>(base + lay.bufB);
  float2* bufC = reinterpret_cast<float2*>(base + lay.bufC);
  const bool pf = A.prefetch != 0;
  float2* tws = reinterpret_cast<float2*>(base + lay.tw);
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

  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) s_sig = atomicAdd(A.work_counter, 1);
    __syncthreads();
    const int qi = s_sig;
    if (qi >= A.batch) break;
    const int b = A.tab.order[qi];
    const int si = A.tab.sig_shape[b];
    if (si != loaded) {
      load_shape(sh, A.tab.shapes, si, tws, A.tab.twiddles, A.tw_smem != 0);
      loaded = si;
    }
    for (int i = threadIdx.x; i < hash_cap; i += blockDim.x) set.hkey[i] = kEmpty;
    if (threadIdx.x == 0) {
      s_count = 0;
      s_ovf = 0;
    }
    __syncthreads();
    const float2* tw = A.tw_smem ? tws : A.tab.twiddles + sh.tw_off;
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
      if (threadIdx.x == 0) s_t0 = 0;
      float2* bins = fft_lines(cur, bufB, D + 1, sh, tw, 1.0f / (float)L);
      peel_set<D>(bins, sh, set, min(s_count, A.k_cap), s_ca, s_ct, tw);
      __syncthreads();
      decode_bins<D>(bins, L, sh, set, s_ca, s_ct, tw, A.th, &s_t0, &s_ovf);
      __syncthreads();
      iters = t + 1;
      const bool stop = (A.early_stop && s_t0 == 0) || s_ovf != 0;
      if (stop) break;
    }

    if (pf) cp_async_wait<0>();   // a prefetch past the last iteration still lands before reuse
    // output: keep |a| > theta0, sorted by linear index (hash arrays reused as sort buffers)
    const int count = min(s_count, A.k_cap);
    sort_kept(set, count, A.th, set.hkey, set.hidx, &s_n);
    const int n = s_n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = set.hidx[r];
#pragma unroll
      for (int d = 0; d < D; ++d) ok_out[r * D + d] = set.lk[d * A.k_cap + i];
      oa_out[r] = set.la[i];
    }
    if (threadIdx.x == 0) {
      A.out_count[b] = n;
      A.out_iters[b] = iters;
      A.out_status[b] = s_ovf ? kStatusCapacity : 0;
    }
    __syncthreads();
  }
}

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

template <int D>
__device__ __forceinline__ void sort_kept_w(const BucketSet& s, const Shape& sh, int count, const Thresholds& th,
                                            int* skey, int* sidx, int* n_out) {
  if (threadIdx.x == 0) *n_out = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    if (keep_amplitude(s.la[i], th)) {
      int key = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) key += s.lk[d * s.k_cap + i] * sh.strides[d];
      const int pos = atomicAdd(n_out, 1);
      skey[pos] = key;
      sidx[pos] = i;
    }
  }
  __syncthreads();
  sort_pairs(skey, sidx, *n_out);
}

// When every bin that passed T0 in iteration t-1 was decoded and merged, the set is most likely
// complete and iteration t will find nothing (the early stop): iteration t then does not prefetch
// t+1.  If the guess is wrong, iteration t+1 gathers its samples synchronously; the results do not
// depend on the guess.
template <int D, int R, bool STAGED>
__device__ __forceinline__ int iterate_w(const RecoverArgs& A, const Shape& sh, const BucketSet& set, float2* bins,
                                         const float2* tws, float2* stg, const float2* __restrict__ x,
                                         const int* sched_a, const int* sched_t, int T, int warp, int lane,
                                         float invL, int* s_ca, int* s_ct, int* s_t0, int* s_ovf, int* s_acc) {
  const int L = sh.L;
  float2 nxt[STAGED ? 1 : R];
  float2* my_stg = stg + warp * L;
  bool have_next = false;      // samples of the current iteration already requested
  bool likely_done = false;    // every T0 bin of the previous iteration was accepted
  if (T > 0) {
    int alr[D], tar[D];
    sched_row<D>(sh, sched_a, sched_t, alr, tar);
    if (STAGED)
      gather_line_async<D, R>(my_stg, x, sh, alr, tar, warp, lane);
    else
      gather_line_regs<D, (STAGED ? 1 : R)>(nxt, x, sh, alr, tar, warp, lane);
    have_next = true;
  }
  int iters = 0;
  for (int t = 0; t < T; ++t) {
    const int* al = sched_a + t * D;
    const int* ta = sched_t + t * D;
    if (threadIdx.x < D) {
      const int d = threadIdx.x;
      s_ca[d] = cmodL(sh, d, al[d]);
      s_ct[d] = cmodL(sh, d, ta[d]);
    }
    for (int m = threadIdx.x; m < L; m += blockDim.x) set.head[m] = -1;
    float2 v[R];
    if (!have_next) {
      int alr[D], tar[D];
      sched_row<D>(sh, al, ta, alr, tar);
      gather_line_regs<D, R>(v, x, sh, alr, tar, warp, lane);
    } else if (STAGED) {
      cp_async_wait<0>();
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = my_stg[lane + 32 * i];
    } else {
#pragma unroll
      for (int i = 0; i < R; ++i) v[i] = nxt[STAGED ? 0 : i];
    }
    fft_store_w<D, R>(v, bins, sh, tws, warp, lane, invL);    // consumes v: the reads above are done
    have_next = t + 1 < T && !likely_done;
    if (have_next) {
      int alr[D], tar[D];
      sched_row<D>(sh, al + D, ta + D, alr, tar);
      if (STAGED)
        gather_line_async<D, R>(my_stg, x, sh, alr, tar, warp, lane);
      else
        gather_line_regs<D, (STAGED ? 1 : R)>(nxt, x, sh, alr, tar, warp, lane);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *s_t0 = 0;
      *s_acc = 0;
    }
    peel_set_w<D>(bins, sh, set, min(*set.count, A.k_cap), s_ca, s_ct, tws);
    __syncthreads();
    decode_bins_w<D>(bins, sh, set, s_ca, s_ct, tws, A.th, s_t0, s_ovf, s_acc);
    __syncthreads();
    iters = t + 1;
    const bool stop = (A.early_stop && *s_t0 == 0) || *s_ovf != 0;
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
#define FPSSFT_WS_THREADS_PER_SM 768   // same for the variant that stages the prefetch in shared memory
#endif

template <int D, bool STAGED>
__global__ void __launch_bounds__(32 * (D + 1), (STAGED ? FPSSFT_WS_THREADS_PER_SM : FPSSFT_W_THREADS_PER_SM) / (32 * (D + 1)))
    k_recover_w(RecoverArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_sig, s_count, s_t0, s_ovf, s_n, s_acc;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
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

  int loaded = -1;
  for (;;) {
    if (threadIdx.x == 0) s_sig = atomicAdd(A.work_counter, 1);
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
      case 1: iters = iterate_w<D, 1, STAGED>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      case 2: iters = iterate_w<D, 2, STAGED>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      case 4: iters = iterate_w<D, 4, STAGED>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
      default: iters = iterate_w<D, 8, STAGED>(A, sh, set, bins, tws, stg, x, sched_a, sched_t, T, warp, lane, invL, s_ca, s_ct, &s_t0, &s_ovf, &s_acc); break;
    }

    const int count = min(s_count, A.k_cap);
    int* skey = reinterpret_cast<int*>(bins);
    int* sidx = skey + (lay.tw - lay.bins) / (2 * sizeof(int));
    sort_kept_w<D>(set, sh, count, A.th, skey, sidx, &s_n);
    const int n = s_n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = sidx[r];
#pragma unroll
      for (int d = 0; d < D; ++d) ok_out[r * D + d] = set.lk[d * A.k_cap + i];
      oa_out[r] = set.la[i];
    }
    if (threadIdx.x == 0) {
      A.out_count[b] = n;
      A.out_iters[b] = iters;
      A.out_status[b] = s_ovf ? kStatusCapacity : 0;
    }
    __syncthreads();
  }
}

// ---- cluster path: one CTA per line, the D+1 CTAs of a signal form a thread-block cluster -------
// For long lines one CTA per signal runs the D+1 transforms one after another on one SM and leaves
// most SMs idle when the batch is small.  Here CTA j of the signal's cluster gathers, transforms
// and peels line j alone in its own shared memory.  Deciding bin m needs bin m of every line, so
// each CTA decodes a (D+1)-th of the bins and reads the other lines' bins through distributed
// shared memory.  The recovered list (key, a) is replicated in every CTA, so each peel reads only
// local memory (k is recovered from the row-major key); the open-addressing index that
// deduplicates keys is split into D+1 contiguous slices, one per rank, and the entry counter is
// rank 0's.  An insert claims its slot wherever it lies and writes the entry into every replica.
// Two cluster barriers per iteration: after the peel (every line's bins final) and after the
// decode (every replica final).  Per CTA: one line, its FFT partner and the prefetch buffer (each
// with room for fft_line's padding), the twiddles and the per-stage twiddles, 12 bytes per set
// entry and 8 bytes per index slot / (D+1).
// GS variant, for sets too large for that: one copy of the list, the whole index and the counter
// live in a per-signal slice of global workspace (cluster_gset_stride bytes), read through L2
// (ld.global.cg: lines written by other SMs are never served from a stale L1 copy); shared memory
// holds only the line buffers and twiddles.
struct CLayout {
  size_t bufA, bufB, bufC, tw, stw, sort, la, lkey, hkey, hidx, total;
  int hc;   // index slots per rank
};

static __host__ __device__ size_t cluster_gset_stride(int k_cap, int hash_cap) {
  const size_t b = (size_t)k_cap * (sizeof(float2) + sizeof(int)) + (size_t)hash_cap * 2 * sizeof(int) + sizeof(int);
  return (b + 255) & ~size_t(255);
}

static __host__ __device__ CLayout recover_layout_c(int D, int L_max, int k_cap, int hash_cap, bool prefetch,
                                                    bool gset = false) {
  auto al = [](size_t v) -> size_t { return (v + 15) & ~size_t(15); };
  CLayout s{};
  const size_t line = (size_t)L_max * sizeof(float2);
  const size_t pline = ((size_t)L_max + (size_t)(L_max - 1) / 16 + 1) * sizeof(float2);   // padq(L - 1) + 1
  size_t P = 1;
  while (P < (size_t)k_cap) P <<= 1;
  s.hc = (hash_cap + D) / (D + 1);
  size_t off = 0;
  s.bufA = off; off = al(off + pline);
  s.bufB = off; off = al(off + pline);
  s.bufC = off; off = al(off + (prefetch ? pline : 0));
  s.tw = off; off = al(off + line);
  s.stw = off; off = al(off + line);
  if (gset) {   // the set, and the output sort's buffers, are in global workspace
    s.sort = s.la = s.lkey = s.hkey = s.hidx = off;
    s.total = off;
    return s;
  }
  // the output sort (rank 0, after the last barrier) reuses the line buffers: 2 P ints
  s.sort = 0;
  const size_t sort_bytes = al(2 * P * sizeof(int));
  if (off < sort_bytes) off = sort_bytes;
  s.la = off; off = al(off + (size_t)k_cap * sizeof(float2));
  s.lkey = off; off = al(off + (size_t)k_cap * sizeof(int));
  s.hkey = off; off = al(off + (size_t)s.hc * sizeof(int));
  s.hidx = off; off = al(off + (size_t)s.hc * sizeof(int));
  s.total = off;
  return s;
}

// Frequency components of a row-major linear index (key < N).
template <int D>
__device__ __forceinline__ void key_to_k(const Shape& sh, int key, int* k) {
#pragma unroll
  for (int d = D - 1; d >= 0; --d) {
    const int q = fdiv(key, sh.fdims[d]);
    k[d] = key - q * sh.dims[d];
    key = q;
  }
}

// a5 from any CTA of the cluster: index slot h lives in rank h / hc at h mod hc, the counter is
// rank 0's, base[r] is rank r's shared memory.  Same contract as set_insert: within one iteration
// concurrent calls carry distinct keys, and an existing key was written in an earlier iteration
// (made visible by the cluster barriers).  Returns false on overflow.
template <int D>
__device__ __forceinline__ bool cluster_insert(unsigned char* const* base, const CLayout& lay, int* count, int k_cap,
                                               int hash_bits, int rank, int key, float2 a) {
  const unsigned mask = (1u << hash_bits) - 1u;
  unsigned h = hash_slot(key, hash_bits);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int r = (int)(h / (unsigned)lay.hc);
    const int i = (int)(h - (unsigned)r * (unsigned)lay.hc);
    int* hkey = reinterpret_cast<int*>(base[r] + lay.hkey);
    int* hidx = reinterpret_cast<int*>(base[r] + lay.hidx);
    const int old = atomicCAS(&hkey[i], kEmpty, key);
    if (old == kEmpty) {
      const int idx = atomicAdd(count, 1);
      if (idx >= k_cap) {
        hidx[i] = -1;
        return false;
      }
#pragma unroll
      for (int q = 0; q <= D; ++q) {
        reinterpret_cast<int*>(base[q] + lay.lkey)[idx] = key;
        reinterpret_cast<float2*>(base[q] + lay.la)[idx] = a;
      }
      hidx[i] = idx;
      return true;
    }
    if (old == key) {
      const int idx = hidx[i];
      if (idx < 0 || idx >= k_cap) return false;   // overflowed claim (or a repeated resume key)
      // every replica holds the same value: add once, write everywhere
      const float2 s = cadd(reinterpret_cast<const float2*>(base[rank] + lay.la)[idx], a);
#pragma unroll
      for (int q = 0; q <= D; ++q) reinterpret_cast<float2*>(base[q] + lay.la)[idx] = s;
      return true;
    }
    h = (h + 1u) & mask;
  }
  return false;   // unreachable at load factor <= 1/2
}

// a5 of the GS variant: the same contract with one global copy of the list, index and counter.
template <int D>
__device__ __forceinline__ bool cluster_insert_g(float2* g_la, int* g_lkey, int* g_hkey, int* g_hidx, int* g_count,
                                                 int k_cap, int hash_bits, int key, float2 a) {
  const unsigned mask = (1u << hash_bits) - 1u;
  unsigned h = hash_slot(key, hash_bits);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int old = atomicCAS(&g_hkey[h], kEmpty, key);
    if (old == kEmpty) {
      const int idx = atomicAdd(g_count, 1);
      if (idx >= k_cap) {
        g_hidx[h] = -1;
        return false;
      }
      g_lkey[idx] = key;
      g_la[idx] = a;
      g_hidx[h] = idx;
      return true;
    }
    if (old == key) {
      const int idx = __ldcg(&g_hidx[h]);
      if (idx < 0 || idx >= k_cap) return false;   // overflowed claim (or a repeated resume key)
      g_la[idx] = cadd(__ldcg(&g_la[idx]), a);
      return true;
    }
    h = (h + 1u) & mask;
  }
  return false;   // unreachable at load factor <= 1/2
}

// Peel of line j from the (key, a) list: entry i lands in bin m with phase p (j = 0) or
// p + c_{j-1} k_{j-1}.  L2ONLY: the list is read through L2 (global list of the GS variant).
template <int D, bool L2ONLY>
__device__ __forceinline__ void peel_line_keys(float2* bins, const Shape& sh, const float2* la, const int* lkey,
                                               int count, const int* ca, const int* ct,
                                               const float2* __restrict__ tw, int j) {
  const int L = sh.L;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    int k[D];
    key_to_k<D>(sh, L2ONLY ? __ldcg(lkey + i) : lkey[i], k);
    int msum = 0, psum = 0, shift = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      msum += ca[d] * k[d];
      psum += ct[d] * k[d];
      if (d == j - 1) shift = sh.c[d] * k[d];
    }
    const int m = fmod_(msum, sh.fL);
    int q = fmod_(psum, sh.fL) + shift;
    if (q >= L) q -= L;
    const float2 v = cmulc(L2ONLY ? __ldcg(la + i) : la[i], tw[q]);
    atomicAdd(&bins[m].x, -v.x);
    atomicAdd(&bins[m].y, -v.y);
  }
}

// One signal per cluster (grid = batch clusters of D+1 CTAs, in the longest-first order).
template <int D, int MAXT, bool GS>
__global__ void __launch_bounds__(MAXT) k_recover_c(RecoverArgs A) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_count, s_ovf, s_n;
  __shared__ int s_t0[2];                     // line-0 bins passing T0, by iteration parity
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  __shared__ unsigned char* s_base[kMaxD + 1];  // each rank's dynamic shared memory (generic address)

  const int rank = (int)cluster.block_rank();
  const int b = A.tab.order[blockIdx.x / (D + 1)];
  const int si = A.tab.sig_shape[b];
  const bool pf = A.prefetch != 0;
  const int hash_cap = 1 << A.hash_bits;
  const CLayout lay = recover_layout_c(D, A.L_max, A.k_cap, hash_cap, pf, GS);
  float2* bufA = reinterpret_cast<float2*>(smem + lay.bufA);
  float2* bufB = reinterpret_cast<float2*>(smem + lay.bufB);
  float2* bufC = reinterpret_cast<float2*>(smem + lay.bufC);
  float2* tws = reinterpret_cast<float2*>(smem + lay.tw);
  float2* stws = reinterpret_cast<float2*>(smem + lay.stw);
  // GS: this signal's slice of global workspace holds the list, the index and the counter
  unsigned char* ws = GS ? A.gm_ws + (size_t)(blockIdx.x / (D + 1)) * A.gm_stride : nullptr;
  float2* g_la = reinterpret_cast<float2*>(ws);
  int* g_lkey = reinterpret_cast<int*>(ws + (size_t)A.k_cap * sizeof(float2));
  int* g_hkey = g_lkey + A.k_cap;
  int* g_hidx = g_hkey + hash_cap;
  int* g_count = g_hidx + hash_cap;
  const float2* la = GS ? g_la : reinterpret_cast<const float2*>(smem + lay.la);
  const int* lkey = GS ? g_lkey : reinterpret_cast<const int*>(smem + lay.lkey);

  load_shape(sh, A.tab.shapes, si, tws, A.tab.twiddles, true);
  {
    const int L = A.tab.shapes[si].L;
    const float2* t = A.tab.twiddles + A.tab.shapes[si].stw_off;
    for (int i = threadIdx.x; i < L - 1; i += blockDim.x) stws[i] = t[i];
  }
  if (threadIdx.x <= D) s_base[threadIdx.x] = cluster.map_shared_rank(smem, (int)threadIdx.x);
  if (GS) {   // every rank clears a (D+1)-th of the global index
    const int hcs = (hash_cap + D) / (D + 1);
    const int h1 = min(hash_cap, (rank + 1) * hcs);
    for (int i = rank * hcs + threadIdx.x; i < h1; i += blockDim.x) g_hkey[i] = kEmpty;
    if (rank == 0 && threadIdx.x == 0) *g_count = 0;
  } else {
    int* hk = reinterpret_cast<int*>(smem + lay.hkey);
    for (int i = threadIdx.x; i < lay.hc; i += blockDim.x) hk[i] = kEmpty;
  }
  if (threadIdx.x == 0) {
    s_count = 0;
    s_ovf = 0;
    s_t0[0] = 0;
    s_t0[1] = 0;
  }
  cluster.sync();   // every CTA started and initialised before any remote access

  int* c_count = GS ? g_count : cluster.map_shared_rank(&s_count, 0);
  int* c_ovf = cluster.map_shared_rank(&s_ovf, 0);
  int* c_t0 = cluster.map_shared_rank(s_t0, 0);
  const float2* x = A.cubes + A.offsets[b];
  int* ok_out = A.out_k + (size_t)b * A.k_cap * D;
  float2* oa_out = A.out_a + (size_t)b * A.k_cap;

  if (A.init_count != nullptr) {   // resume from a given set (rank 0 inserts into every replica)
    if (rank == 0) {
      const int n0 = min(max(A.init_count[b], 0), A.k_cap);
      for (int i = threadIdx.x; i < n0; i += blockDim.x) {
        int k[D];
        int key = 0;
#pragma unroll
        for (int d = 0; d < D; ++d) {
          k[d] = ok_out[i * D + d];
          key += k[d] * sh.strides[d];
        }
        const bool ok = !on_grid<D>(sh, k) ||
                        (GS ? cluster_insert_g<D>(g_la, g_lkey, g_hkey, g_hidx, g_count, A.k_cap, A.hash_bits, key, oa_out[i])
                            : cluster_insert<D>(s_base, lay, c_count, A.k_cap, A.hash_bits, rank, key, oa_out[i]));
        if (!ok) atomicOr(c_ovf, 1);
      }
    }
    cluster.sync();
  }
  int n_set = min(GS ? __ldcg(g_count) : *c_count, A.k_cap);
  const bool stop = *c_ovf != 0;

  const int L = sh.L;
  const int chunk = (L + D) / (D + 1);
  const int m_lo = rank * chunk;
  const int m_hi = min(L, m_lo + chunk);
  const int T = stop ? 0 : A.tab.sig_T[b];
  const int* sched_a = A.alpha + (size_t)b * A.sched_stride;
  const int* sched_t = A.tau + (size_t)b * A.sched_stride;
  if (pf && T > 0) gather_one_line<D, 0, true>(bufA, x, sh, sched_a, sched_t, rank);
  int iters = 0;
  for (int t = 0; t < T; ++t) {
    const int par = t & 1;
    const int* al = sched_a + t * D;
    const int* ta = sched_t + t * D;
    // slot par was last read after the decode barrier of iteration t-2, before every rank
    // arrived at the peel barrier of t-1, which this rank has passed
    if (rank == 0 && threadIdx.x == 0) s_t0[par] = 0;
    if (threadIdx.x < D) {
      const int d = threadIdx.x;
      s_ca[d] = cmodL(sh, d, al[d]);
      s_ct[d] = cmodL(sh, d, ta[d]);
    }
    float2* cur = (pf && (t & 1)) ? bufC : bufA;
    if (pf) {
      if (t + 1 < T) {
        gather_one_line<D, 0, true>((t & 1) ? bufA : bufC, x, sh, al + D, ta + D, rank);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
    } else if (A.gather_mode == 2) {
      gather_one_line<D, 1, false>(bufA, x, sh, al, ta, rank);
    } else {
      gather_one_line<D, 0, false>(bufA, x, sh, al, ta, rank);
    }
    __syncthreads();
    float2* bins = fft_line(cur, bufB, sh, tws, stws, 1.0f / (float)L);
    peel_line_keys<D, GS>(bins, sh, la, lkey, n_set, s_ca, s_ct, tws, rank);
    cluster.sync();   // every line peeled

    const size_t boff = reinterpret_cast<unsigned char*>(bins) - smem;
    int my_t0 = 0;
    bool my_ovf = false;
    for (int m = m_lo + threadIdx.x; m < m_hi; m += blockDim.x) {
      const float2 s0 = reinterpret_cast<const float2*>(s_base[0] + boff)[m];
      float2 sd[D];
#pragma unroll
      for (int d = 0; d < D; ++d) sd[d] = reinterpret_cast<const float2*>(s_base[d + 1] + boff)[m];
      int k[D];
      bool counted = false;
      int v = A.th.fp64_all ? kUndecided : classify_fp32<D>(s0, sd, sh, A.th, k, &counted);
      if (v == kUndecided) {
        bool c64 = false;
        v = classify_fp64<D>(s0, sd, sh, A.th, k, &c64);
        counted = c64;
      }
      my_t0 += counted ? 1 : 0;
      if (v != kAccept) continue;
      int msum = 0, psum = 0, key = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        msum += s_ca[d] * k[d];
        psum += s_ct[d] * k[d];
        key += k[d] * sh.strides[d];
      }
      if (fmod_(msum, sh.fL) != m) continue;                            // T3
      const float2 a = decoded_amplitude<D>(s0, sd, sh, k, fmod_(psum, sh.fL), tws, A.th.amp_average != 0);
      const bool ok = GS ? cluster_insert_g<D>(g_la, g_lkey, g_hkey, g_hidx, g_count, A.k_cap, A.hash_bits, key, a)
                         : cluster_insert<D>(s_base, lay, c_count, A.k_cap, A.hash_bits, rank, key, a);
      if (!ok) my_ovf = true;
    }
    if (my_t0) atomicAdd(c_t0 + par, my_t0);
    if (my_ovf) atomicOr(c_ovf, 1);
    cluster.sync();   // every insert landed in every replica
    n_set = min(GS ? __ldcg(g_count) : *c_count, A.k_cap);
    iters = t + 1;
    if ((A.early_stop && c_t0[par] == 0) || *c_ovf != 0) break;   // the same verdict on every rank
  }
  if (pf) cp_async_wait<0>();
  cluster.sync();   // no rank reads another's shared memory past this point

  if (rank != 0) return;
  // output order: a bitmap of the grid points in the shared memory the set does not use (all of it
  // with GS), else sorted (key, position) pairs
  {
    auto get = [&](int i, int& key, float2& a) -> bool {
      a = GS ? __ldcg(la + i) : la[i];
      if (!keep_amplitude(a, A.th)) return false;
      key = GS ? __ldcg(lkey + i) : lkey[i];
      return true;
    };
    auto put = [&](int r, int key, float2 a) {
      int k[D];
      key_to_k<D>(sh, key, k);
#pragma unroll
      for (int d = 0; d < D; ++d) ok_out[r * D + d] = k[d];
      oa_out[r] = a;
    };
    if (emit_by_bitmap(n_set, sh.N, smem, GS ? lay.total : lay.la, &s_n, get, put)) {
      if (threadIdx.x == 0) {
        A.out_count[b] = s_n;
        A.out_iters[b] = iters;
        A.out_status[b] = s_ovf ? kStatusCapacity : 0;
      }
      return;
    }
  }
  int P = 1;
  while (P < A.k_cap) P <<= 1;
  // sort buffers: the line buffers, free now, or (GS) the global index
  int* skey = GS ? g_hkey : reinterpret_cast<int*>(smem + lay.sort);
  int* sidx = GS ? g_hidx : skey + P;
  if (threadIdx.x == 0) s_n = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n_set; i += blockDim.x) {
    if (keep_amplitude(GS ? __ldcg(la + i) : la[i], A.th)) {
      const int pos = atomicAdd(&s_n, 1);
      skey[pos] = GS ? __ldcg(lkey + i) : lkey[i];
      sidx[pos] = i;
    }
  }
  __syncthreads();
  const int n = s_n;
  sort_pairs(skey, sidx, n);
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const int i = sidx[r];
    int k[D];
    key_to_k<D>(sh, skey[r], k);
#pragma unroll
    for (int d = 0; d < D; ++d) ok_out[r * D + d] = k[d];
    oa_out[r] = GS ? __ldcg(la + i) : la[i];
  }
  if (threadIdx.x == 0) {
    A.out_count[b] = n;
    A.out_iters[b] = iters;
    A.out_status[b] = s_ovf ? kStatusCapacity : 0;
  }
}

// ---- projection / raw lines: one CTA per (signal, schedule row) --------------------------------
struct ProjectArgs {
  const float2* cubes;
  const int64_t* offsets;
  const int* alpha;
  const int* tau;
  int n_sched;
  DeviceTables tab;
  int batch;
  int L_max;
  int dft;
  float2* out;      // [batch][n_sched][D+1][L_max]
};

template <int D>
__global__ void __launch_bounds__(256) k_project(ProjectArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  float2* bufA = reinterpret_cast<float2*>(smem);
  float2* bufB = bufA + (size_t)(D + 1) * A.L_max;
  int loaded = -1;
  const long long units = (long long)A.batch * A.n_sched;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int b = (int)(u / A.n_sched);
    const int si = A.tab.sig_shape[b];
    if (si != loaded) {
      __syncthreads();
      load_shape(sh, A.tab.shapes, si, nullptr, A.tab.twiddles, false);
      loaded = si;
      __syncthreads();
    }
    const int L = sh.L;
    const int* al = A.alpha + u * D;
    const int* ta = A.tau + u * D;
    gather_lines<D>(bufA, A.cubes + A.offsets[b], sh, al, ta);
    __syncthreads();
    const float2* res = A.dft ? fft_lines(bufA, bufB, D + 1, sh, A.tab.twiddles + sh.tw_off, 1.0f / (float)L) : bufA;
    float2* o = A.out + u * (D + 1) * (long long)A.L_max;
    for (int i = threadIdx.x; i < (D + 1) * A.L_max; i += blockDim.x) {
      const int j = i / A.L_max, m = i - j * A.L_max;
      o[i] = (m < L) ? res[j * L + m] : make_float2(0.f, 0.f);
    }
    __syncthreads();
  }
}

// ---- synthesis (+, overwrite / accumulate) and peel (-) ------------------------------------------
struct SynthArgs {
  const int* alpha;
  const int* tau;
  int n_sched;
  DeviceTables tab;
  int batch;
  int L_max;
  int k_cap;
  const int* k;
  const float2* a;
  const int* count;
  int accumulate;   // 0 overwrite, +1 add, -1 subtract
  float2* bins;
};

template <int D>
__global__ void __launch_bounds__(256) k_synth(SynthArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  float2* acc = reinterpret_cast<float2*>(smem);
  int loaded = -1;
  const long long units = (long long)A.batch * A.n_sched;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int b = (int)(u / A.n_sched);
    const int si = A.tab.sig_shape[b];
    __syncthreads();
    if (si != loaded) {
      load_shape(sh, A.tab.shapes, si, nullptr, A.tab.twiddles, false);
      loaded = si;
      __syncthreads();
    }
    const int L = sh.L;
    const int* al = A.alpha + u * D;
    const int* ta = A.tau + u * D;
    if (threadIdx.x < D) {
      const int d = threadIdx.x;
      s_ca[d] = cmodL(sh, d, al[d]);
      s_ct[d] = cmodL(sh, d, ta[d]);
    }
    float2* o = A.bins + u * (D + 1) * (long long)A.L_max;
    for (int i = threadIdx.x; i < (D + 1) * L; i += blockDim.x) {
      const int j = i / L, m = i - j * L;
      acc[i] = A.accumulate ? o[j * A.L_max + m] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    const float sign = A.accumulate < 0 ? -1.f : 1.f;
    const int cnt = min(max(A.count[b], 0), A.k_cap);
    const float2* tw = A.tab.twiddles + sh.tw_off;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      int k[D];
#pragma unroll
      for (int d = 0; d < D; ++d) k[d] = A.k[((size_t)b * A.k_cap + i) * D + d];
      if (on_grid<D>(sh, k)) project_entry<D>(acc, L, sh, k, A.a[(size_t)b * A.k_cap + i], s_ca, s_ct, tw, sign);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < (D + 1) * A.L_max; i += blockDim.x) {
      const int j = i / A.L_max, m = i - j * A.L_max;
      o[i] = (m < L) ? acc[j * L + m] : make_float2(0.f, 0.f);
    }
  }
}

// ---- one iteration's decode + merge on bins in global memory (unfused form) ----------------------
struct DecodeArgs {
  const float2* bins;   // [batch][1][D+1][L_max]
  const int* alpha;
  const int* tau;
  DeviceTables tab;
  int batch;
  int L_max;
  int k_cap;
  int hash_bits;
  Thresholds th;
  int* k;
  float2* a;
  int* count;
  int* t0_count;
  int* status;
};

template <int D>
__global__ void __launch_bounds__(256) k_decode(DecodeArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_count, s_t0, s_ovf;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  const int hash_cap = 1 << A.hash_bits;
  SetView set;
  set.la = reinterpret_cast<float2*>(smem);
  set.lk = reinterpret_cast<int*>(set.la + A.k_cap);
  set.lkey = set.lk + (size_t)D * A.k_cap;
  set.hkey = set.lkey + A.k_cap;
  set.hidx = set.hkey + hash_cap;
  set.count = &s_count;
  set.k_cap = A.k_cap;
  set.hash_bits = A.hash_bits;
  for (int b = blockIdx.x; b < A.batch; b += gridDim.x) {
    __syncthreads();
    load_shape(sh, A.tab.shapes, A.tab.sig_shape[b], nullptr, A.tab.twiddles, false);
    for (int i = threadIdx.x; i < hash_cap; i += blockDim.x) set.hkey[i] = kEmpty;
    if (threadIdx.x == 0) {
      s_count = 0;
      s_t0 = 0;
      s_ovf = 0;
    }
    __syncthreads();
    if (threadIdx.x < D) {
      const int d = threadIdx.x;
      s_ca[d] = cmodL(sh, d, A.alpha[b * D + d]);
      s_ct[d] = cmodL(sh, d, A.tau[b * D + d]);
    }
    const int n0 = min(max(A.count[b], 0), A.k_cap);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      int k[D];
      int key = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        k[d] = A.k[((size_t)b * A.k_cap + i) * D + d];
        key += k[d] * sh.strides[d];
      }
      if (on_grid<D>(sh, k)) set_insert<D>(set, k, key, A.a[(size_t)b * A.k_cap + i]);
    }
    __syncthreads();
    decode_bins<D>(A.bins + (size_t)b * (D + 1) * A.L_max, A.L_max, sh, set, s_ca, s_ct,
                   A.tab.twiddles + sh.tw_off, A.th, &s_t0, &s_ovf);
    __syncthreads();
    const int cnt = min(s_count, A.k_cap);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
#pragma unroll
      for (int d = 0; d < D; ++d) A.k[((size_t)b * A.k_cap + i) * D + d] = set.lk[d * A.k_cap + i];
      A.a[(size_t)b * A.k_cap + i] = set.la[i];
    }
    if (threadIdx.x == 0) {
      A.count[b] = cnt;
      A.t0_count[b] = s_t0;
      if (s_ovf) A.status[b] |= kStatusCapacity;
    }
  }
}

// ---- finalize: drop small amplitudes and sort (unfused form) -------------------------------------
struct FinalizeArgs {
  DeviceTables tab;
  int batch;
  int k_cap;
  int sort_cap;     // power of two >= k_cap
  Thresholds th;
  int* k;
  float2* a;
  int* count;
};

template <int D>
__global__ void __launch_bounds__(256) k_finalize(FinalizeArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_n;
  SetView set;
  set.la = reinterpret_cast<float2*>(smem);
  set.lk = reinterpret_cast<int*>(set.la + A.k_cap);
  set.lkey = set.lk + (size_t)D * A.k_cap;
  int* skey = set.lkey + A.k_cap;
  int* sidx = skey + A.sort_cap;
  set.k_cap = A.k_cap;
  for (int b = blockIdx.x; b < A.batch; b += gridDim.x) {
    __syncthreads();
    load_shape(sh, A.tab.shapes, A.tab.sig_shape[b], nullptr, A.tab.twiddles, false);
    __syncthreads();
    const int n0 = min(max(A.count[b], 0), A.k_cap);
    for (int i = threadIdx.x; i < n0; i += blockDim.x) {
      int key = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        const int kd = A.k[((size_t)b * A.k_cap + i) * D + d];
        set.lk[d * A.k_cap + i] = kd;
        key += kd * sh.strides[d];
      }
      set.lkey[i] = key;
      set.la[i] = A.a[(size_t)b * A.k_cap + i];
    }
    __syncthreads();
    sort_kept(set, n0, A.th, skey, sidx, &s_n);
    const int n = s_n;
    for (int r = threadIdx.x; r < n; r += blockDim.x) {
      const int i = sidx[r];
#pragma unroll
      for (int d = 0; d < D; ++d) A.k[((size_t)b * A.k_cap + r) * D + d] = set.lk[d * A.k_cap + i];
      A.a[(size_t)b * A.k_cap + r] = set.la[i];
    }
    if (threadIdx.x == 0) A.count[b] = n;
  }
}

// ---- adjoints --------------------------------------------------------------------------------
struct AdjProjectArgs {
  const float2* g;         // [batch][n_sched][D+1][L_max]
  const int64_t* offsets;
  const int* alpha;
  const int* tau;
  int n_sched;
  DeviceTables tab;
  int batch;
  int L_max;
  float2* grad;            // cube layout
};

template <int D>
__global__ void __launch_bounds__(256) k_adjoint_project(AdjProjectArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  float2* bufA = reinterpret_cast<float2*>(smem);
  float2* bufB = bufA + (size_t)(D + 1) * A.L_max;
  int loaded = -1;
  const long long units = (long long)A.batch * A.n_sched;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int b = (int)(u / A.n_sched);
    const int si = A.tab.sig_shape[b];
    if (si != loaded) {
      __syncthreads();
      load_shape(sh, A.tab.shapes, si, nullptr, A.tab.twiddles, false);
      loaded = si;
      __syncthreads();
    }
    const int L = sh.L;
    const float2* g = A.g + u * (D + 1) * (long long)A.L_max;
    for (int i = threadIdx.x; i < (D + 1) * L; i += blockDim.x) {
      const int j = i / L, m = i - j * L;
      const float2 v = g[j * A.L_max + m];
      bufA[i] = make_float2(v.x, -v.y);          // conj(g)
    }
    __syncthreads();
    // (1/L) sum_m g(m) exp(+j 2 pi l m / L) = conj( (1/L) DFT(conj g) )
    const float2* res = fft_lines(bufA, bufB, D + 1, sh, A.tab.twiddles + sh.tw_off, 1.0f / (float)L);
    int al[D], ta[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
      al[d] = fmod_(A.alpha[u * D + d] & 0x3fffffff, sh.fdims[d]);
      ta[d] = fmod_(A.tau[u * D + d] & 0x3fffffff, sh.fdims[d]);
    }
    float2* out = A.grad + A.offsets[b];
    for (int i = threadIdx.x; i < (D + 1) * L; i += blockDim.x) {
      const int j = i / L, l = i - j * L;
      const float2 v = res[i];
      const int addr = line_address<D>(sh, al, ta, j, l);
      atomicAdd(&out[addr].x, v.x);
      atomicAdd(&out[addr].y, -v.y);
    }
    __syncthreads();
  }
}

struct AdjSynthArgs {
  const float2* g;         // [batch][n_sched][D+1][L_max]
  const int* alpha;
  const int* tau;
  int n_sched;
  DeviceTables tab;
  int batch;
  int L_max;
  int k_cap;
  const int* k;
  const int* count;
  float2* grad_a;          // [batch][k_cap]
};

template <int D>
__global__ void __launch_bounds__(256) k_adjoint_synth(AdjSynthArgs A) {
  const long long total = (long long)A.batch * A.k_cap;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(t / A.k_cap);
    const int i = (int)(t - (long long)b * A.k_cap);
    if (i >= min(max(A.count[b], 0), A.k_cap)) continue;
    const Shape& sh = A.tab.shapes[A.tab.sig_shape[b]];
    const int L = sh.L;
    const float2* tw = A.tab.twiddles + sh.tw_off;
    int k[D];
#pragma unroll
    for (int d = 0; d < D; ++d) k[d] = A.k[((size_t)b * A.k_cap + i) * D + d];
    float2 acc = make_float2(0.f, 0.f);
    for (int s = 0; s < A.n_sched && on_grid<D>(sh, k); ++s) {
      const long long u = (long long)b * A.n_sched + s;
      long long msum = 0, psum = 0;
#pragma unroll
      for (int d = 0; d < D; ++d) {
        msum += (long long)cmodL(sh, d, A.alpha[u * D + d]) * k[d];
        psum += (long long)cmodL(sh, d, A.tau[u * D + d]) * k[d];
      }
      const int m = (int)(msum % L);
      const int p = (int)(psum % L);
      const float2* g = A.g + u * (D + 1) * (long long)A.L_max;
      acc = cadd(acc, cmul(tw[p], g[m]));      // conj(W^p) = tw[p]
#pragma unroll
      for (int d = 0; d < D; ++d) {
        int q = p + sh.c[d] * k[d];
        if (q >= L) q -= L;
        acc = cadd(acc, cmul(tw[q], g[(d + 1) * A.L_max + m]));
      }
    }
    A.grad_a[(size_t)b * A.k_cap + i] = acc;
  }
}

// ================================================================================================
// Host side: plan
// ================================================================================================

struct fpssft_plan_s {
  int device = 0;
  int D = 0;
  int batch = 0;
  fpssft_params p{};
  int L_max = 1;
  int T_max = 1;
  int hash_bits = 1;
  int n_shapes = 0;
  int threads = 256;
  int grid = 1;
  int sm_count = 1;
  bool tw_smem = true;
  bool prefetch = true;
  bool warp_path = false;   // k_recover_w (register FFT per line) instead of k_recover
  bool gm_path = false;     // k_recover with lines and set in global workspace
  bool cluster_path = false;   // k_recover_c (one CTA per line, a cluster of D+1 CTAs per signal)
  bool cluster_gs = false;     // ... with the recovered set in global workspace (GS variant)
  bool lines_in_smem = true;   // fpssft_project / _lines / _adjoint / _synth usable
  bool set_in_smem = true;     // fpssft_decode / _finalize usable (one signal's set in one CTA)
  unsigned char* d_gm_ws = nullptr;
  size_t gm_stride = 0;
  size_t smem = 0;
  size_t total_elems = 0;   // sum of N_b (for host staging)
  std::vector<Shape> shapes;
  std::vector<int> sig_shape, sig_T, order, sig_L;
  // device workspace
  Shape* d_shapes = nullptr;
  int* d_sig_shape = nullptr;
  int* d_sig_T = nullptr;
  int* d_order = nullptr;
  float2* d_twiddles = nullptr;
  int* d_counter = nullptr;
  // host-call staging (allocated on the first fpssft_recover_host call)
  void* st_cubes = nullptr;
  size_t st_cubes_elems = 0;
  int64_t* st_offsets = nullptr;
  int32_t* st_alpha = nullptr;
  int32_t* st_tau = nullptr;
  int32_t* st_init = nullptr;
  int32_t* st_k = nullptr;
  void* st_a = nullptr;
  int32_t* st_count = nullptr;
  int32_t* st_iters = nullptr;
  int32_t* st_status = nullptr;

  DeviceTables tables() const { return DeviceTables{d_shapes, d_sig_shape, d_sig_T, d_order, d_twiddles}; }
  Thresholds thresholds() const {
    // FP32 guard bands: 1e-6 relative on either side of each FP64 threshold (FP32 evaluation
    // error <= 3e-7 relative), rounded outward to the next float.
    auto up = [](double v) { float f = (float)v; return (double)f < v ? std::nextafter(f, INFINITY) : f; };
    auto down = [](double v) { float f = (float)v; return (double)f > v ? std::nextafter(f, -INFINITY) : f; };
    const double g = 1e-6;
    Thresholds t;
    t.th0sq = (double)p.theta0 * (double)p.theta0;
    t.rho = p.rho;
    t.eta = p.eta;
    t.t0_lo = down(t.th0sq * (1.0 - g));
    t.t0_hi = up(t.th0sq * (1.0 + g));
    const double hi2 = (1.0 + t.rho) * (1.0 + t.rho);
    const double lo = std::max(0.0, 1.0 - t.rho);
    const double lo2 = lo * lo;
    t.t1_hi_pass = down(hi2 * (1.0 - 2 * g));
    t.t1_hi_fail = up(hi2 * (1.0 + 2 * g));
    t.t1_lo_pass = lo2 > 0 ? up(lo2 * (1.0 + 2 * g)) : 0.f;
    t.t1_lo_fail = lo2 > 0 ? down(lo2 * (1.0 - 2 * g)) : -1.f;
    t.eta_f = (float)t.eta;
    t.fp64_all = p.fp64_decisions ? 1 : 0;
    t.amp_average = p.amp_average ? 1 : 0;
    return t;
  }
};

namespace {

FastDiv make_fastdiv(int d) {
  int l = 0;
  while ((1LL << l) < d) ++l;
  const unsigned long long m = ((1ULL << 32) * ((1ULL << l) - (unsigned long long)d)) / (unsigned long long)d + 1ULL;
  FastDiv f;
  f.m = (unsigned)m;
  f.l = l;
  f.d = d;
  f.pad_ = 0;
  return f;
}

std::vector<int> factorize(int L) {
  std::vector<int> r;
  int n = L;
  while (n % 8 == 0) { r.push_back(8); n /= 8; }
  while (n % 4 == 0) { r.push_back(4); n /= 4; }
  while (n % 2 == 0) { r.push_back(2); n /= 2; }
  while (n % 3 == 0) { r.push_back(3); n /= 3; }
  while (n % 5 == 0) { r.push_back(5); n /= 5; }
  for (int f = 7; (long long)f * f <= n; f += 2) {
    while (n % f == 0) { r.push_back(f); n /= f; }
  }
  if (n > 1) r.push_back(n);
  return r;
}

template <typename F>
fpssft_status dispatch_D(int D, F&& f) {
  switch (D) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    default: return fail(FPSSFT_ERR_INVALID, "D must be in [1, 4]");
  }
}

void free_plan_memory(fpssft_plan_s* p) {
  cudaFree(p->d_gm_ws);
  cudaFree(p->d_shapes);
  cudaFree(p->d_sig_shape);
  cudaFree(p->d_sig_T);
  cudaFree(p->d_order);
  cudaFree(p->d_twiddles);
  cudaFree(p->d_counter);
  cudaFree(p->st_cubes);
  cudaFree(p->st_offsets);
  cudaFree(p->st_alpha);
  cudaFree(p->st_tau);
  cudaFree(p->st_init);
  cudaFree(p->st_k);
  cudaFree(p->st_a);
  cudaFree(p->st_count);
  cudaFree(p->st_iters);
  cudaFree(p->st_status);
}

size_t line_smem(int D, int L_max) { return 2 * (size_t)(D + 1) * L_max * sizeof(float2); }

}  // namespace

extern "C" fpssft_status fpssft_plan_create(fpssft_plan_t* out, int D, int batch, const int64_t* dims,
                                            const fpssft_params* params) {
  g_last_error.clear();
  if (out == nullptr || params == nullptr) return fail(FPSSFT_ERR_INVALID, "null out or params");
  *out = nullptr;
  if (D < 1 || D > kMaxD) return fail(FPSSFT_ERR_INVALID, "D must be in [1, 4]");
  if (batch < 0) return fail(FPSSFT_ERR_INVALID, "batch must be >= 0");
  if (batch > 0 && dims == nullptr) return fail(FPSSFT_ERR_INVALID, "null dims");
  const fpssft_params& pr = *params;
  if (pr.k_cap < 1 || pr.k_cap > (1 << 22)) return fail(FPSSFT_ERR_INVALID, "k_cap must be in [1, 2^22]");
  if (pr.T < 0) return fail(FPSSFT_ERR_INVALID, "T must be >= 0");
  if (!(pr.theta0 >= 0.f) || !(pr.rho >= 0.f) || !(pr.eta >= 0.f)) return fail(FPSSFT_ERR_INVALID, "thresholds must be >= 0");
  if (pr.peel_mode != 0) return fail(FPSSFT_ERR_UNSUPPORTED, "only peel_mode 0 (bins) is implemented on the GPU");
  if (pr.gather_mode < 0 || pr.gather_mode > 3) return fail(FPSSFT_ERR_INVALID, "gather_mode must be in [0, 3]");
  if (pr.fft_path < 0 || pr.fft_path > 3) return fail(FPSSFT_ERR_INVALID, "fft_path must be in [0, 3]");
  if (pr.threads < 0 || pr.threads > 1024 || (pr.threads % 32) != 0) return fail(FPSSFT_ERR_INVALID, "threads must be a multiple of 32 in [0, 1024]");

  auto* P = new (std::nothrow) fpssft_plan_s();
  if (!P) return fail(FPSSFT_ERR_ALLOC, "host allocation failed");
  P->D = D;
  P->batch = batch;
  P->p = pr;
  cudaGetDevice(&P->device);

  std::map<std::vector<int>, int> shape_id;
  std::map<int, int> tw_off;
  std::vector<float2> tw_pool;
  P->sig_shape.resize(batch);
  P->sig_T.resize(batch);
  P->sig_L.resize(batch);
  size_t total = 0;
  for (int b = 0; b < batch; ++b) {
    std::vector<int> dv(D);
    long long N = 1, L = 1, nmax = 1;
    for (int d = 0; d < D; ++d) {
      const int64_t n = dims[(size_t)b * D + d];
      if (n < 1 || n > (1 << 24)) { delete P; return fail(FPSSFT_ERR_INVALID, "every dimension must be in [1, 2^24]"); }
      dv[d] = (int)n;
      N *= n;
      L = L / std::gcd(L, (long long)n) * n;
      nmax = std::max(nmax, (long long)n);
      if (N > (1LL << 31) - 1 || L > (1LL << 24)) { delete P; return fail(FPSSFT_ERR_UNSUPPORTED, "cube or line too large (N < 2^31, L <= 2^24)"); }
    }
    if ((long long)D * L * nmax >= (1LL << 31)) { delete P; return fail(FPSSFT_ERR_UNSUPPORTED, "D * L * max N_d must stay below 2^31"); }
    total += (size_t)N;
    auto it = shape_id.find(dv);
    int si;
    if (it == shape_id.end()) {
      Shape sh{};
      sh.D = D;
      sh.L = (int)L;
      sh.N = (int)N;
      int stride = 1;
      for (int d = D - 1; d >= 0; --d) { sh.dims[d] = dv[d]; sh.strides[d] = stride; stride *= dv[d]; }
      for (int d = 0; d < D; ++d) sh.c[d] = (int)(L / dv[d]);
      auto rad = factorize((int)L);
      if ((int)rad.size() > kMaxStages) { delete P; return fail(FPSSFT_ERR_UNSUPPORTED, "too many FFT stages"); }
      sh.nst = (int)rad.size();
      for (int d = 0; d < kMaxD; ++d) sh.fdims[d] = make_fastdiv(d < D ? dv[d] : 1);
      sh.fL = make_fastdiv((int)L);
      int ns = 1;
      for (size_t s = 0; s < rad.size(); ++s) {
        sh.radix[s] = rad[s];
        sh.tstep[s] = (int)(L / ((long long)ns * rad[s]));
        sh.fnb[s] = make_fastdiv((int)(L / rad[s]));
        sh.fns[s] = make_fastdiv(ns);
        ns *= rad[s];
      }
      auto t = tw_off.find((int)L);
      if (t == tw_off.end()) {
        const int off = (int)tw_pool.size();
        tw_off[(int)L] = off;
        for (long long q = 0; q < L; ++q) {
          // exp(-j 2 pi q / L) in FP64, rounded to FP32
          const double ang = 2.0 * M_PI * (double)q / (double)L;
          tw_pool.push_back(make_float2((float)std::cos(ang), (float)-std::sin(ang)));
        }
        // per-stage table of the one-line FFT: entry i Ns + k - 1 = exp(-j 2 pi i k tstep / L)
        std::vector<float2> stw((size_t)std::max(0LL, L - 1));
        for (int st = 0, nss = 1; st < sh.nst; nss *= sh.radix[st], ++st)
          for (int i = 1; i < sh.radix[st]; ++i)
            for (int k = 0; k < nss; ++k)
              stw[(size_t)i * nss + k - 1] = tw_pool[off + (size_t)i * k * sh.tstep[st]];
        tw_pool.insert(tw_pool.end(), stw.begin(), stw.end());
        sh.tw_off = off;
      } else {
        sh.tw_off = t->second;
      }
      sh.stw_off = sh.tw_off + (int)L;
      si = (int)P->shapes.size();
      shape_id[dv] = si;
      P->shapes.push_back(sh);
    } else {
      si = it->second;
    }
    P->sig_shape[b] = si;
    P->sig_L[b] = (int)L;
    const long long budget = std::max(1LL, N / ((long long)(D + 1) * L));
    P->sig_T[b] = pr.T > 0 ? pr.T : (int)std::min(budget, (long long)1 << 30);
    P->L_max = std::max(P->L_max, (int)L);
    P->T_max = std::max(P->T_max, P->sig_T[b]);
  }
  P->total_elems = total;
  P->n_shapes = (int)P->shapes.size();
  // longest lines first, then the larger iteration budget (longest-processing-time order)
  P->order.resize(batch);
  std::iota(P->order.begin(), P->order.end(), 0);
  std::stable_sort(P->order.begin(), P->order.end(), [&](int a, int b) {
    if (P->sig_L[a] != P->sig_L[b]) return P->sig_L[a] > P->sig_L[b];
    return P->sig_T[a] > P->sig_T[b];
  });
  int hb = 1;
  while ((1 << hb) < 2 * pr.k_cap) ++hb;
  P->hash_bits = hb;

  int dev = P->device;
  int optin = 0, sms = 1;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (optin <= 0) optin = 227 * 1024;
  if (sms <= 0) sms = 1;
  P->sm_count = sms;
  const size_t static_reserve = sizeof(Shape) + 256;
  // the register-FFT path applies when every line length is 32 R with R in {1, 2, 4, 8}
  bool warp_ok = true;
  for (const Shape& sh : P->shapes) {
    const int R = sh.L / 32;
    warp_ok = warp_ok && sh.L % 32 == 0 && (R == 1 || R == 2 || R == 4 || R == 8);
  }
  warp_ok = warp_ok && pr.k_cap < (1 << 20);
  if (pr.fft_path == 2 && !warp_ok) {
    delete P;
    return fail(FPSSFT_ERR_UNSUPPORTED, "fft_path 2 needs every line length in {32, 64, 128, 256} and no prefetch");
  }
  if ((pr.fft_path == 2 || (pr.fft_path == 0 && warp_ok)) && batch > 0) {
    const WLayout wl = recover_layout_w(D, P->L_max, pr.k_cap, pr.gather_mode == 3);
    if (wl.total + sizeof(Shape) + 256 <= (size_t)optin) {
      P->warp_path = true;
      P->smem = wl.total;
      P->tw_smem = true;
      P->prefetch = pr.gather_mode == 3;   // staged in shared memory by cp.async
      P->threads = 32 * (D + 1);
    } else if (pr.fft_path == 2) {
      delete P;
      return fail(FPSSFT_ERR_UNSUPPORTED, "lines + recovered set exceed one CTA's shared memory (k_cap too large)");
    }
  }
  const bool want_pf = pr.gather_mode == 3;
  if (pr.fft_path == 3 && batch > (1 << 28)) {
    delete P;
    return fail(FPSSFT_ERR_UNSUPPORTED, "fft_path 3 launches batch (D+1) CTAs: batch must be <= 2^28");
  }
  // library choice: long lines and no more signals than twice the SM count go to the cluster
  // path when it fits (one CTA per signal would leave SMs idle and run the lines one by one)
  const bool cluster_auto = pr.fft_path == 0 && !P->warp_path && P->L_max >= 1024 && batch <= 2 * sms &&
                            recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, false, true).total + static_reserve <= (size_t)optin;
  if ((pr.fft_path == 3 || cluster_auto) && batch > 0) {
    // one line, its FFT partner, the twiddles and a replica of the recovered list per CTA.  The
    // library's choice (measured on 240 x 256 and 1024^2): lines of 2048 or more with 1024-thread
    // CTAs and synchronous gathers, shorter lines with 512 threads and the next iteration's line
    // prefetched
    const bool pf_c = pr.gather_mode == 3 || (pr.gather_mode == 0 && P->L_max < 2048);
    // the set in shared memory if it fits (with, then without the prefetch buffer), else in
    // global workspace
    const size_t cap = (size_t)optin - static_reserve;
    bool gs = false;
    CLayout cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, pf_c);
    P->prefetch = pf_c;
    if (cl.total > cap && pf_c) {
      cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, false);
      P->prefetch = false;
    }
    if (cl.total > cap) {
      gs = true;
      cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, pf_c, true);
      P->prefetch = pf_c;
      if (cl.total > cap && pf_c) {
        cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, false, true);
        P->prefetch = false;
      }
    }
    if (cl.total > cap) {
      delete P;
      return fail(FPSSFT_ERR_UNSUPPORTED, "fft_path 3: one line and its twiddles exceed one CTA's shared memory");
    }
    P->cluster_path = true;
    P->cluster_gs = gs;
    if (gs) P->gm_stride = cluster_gset_stride(pr.k_cap, 1 << hb);
    P->tw_smem = true;
    P->smem = cl.total;
    if (pr.threads > 0) {
      P->threads = pr.threads;
    } else if (P->L_max >= 2048) {
      P->threads = 1024;
    } else {
      int t = 128;
      while (2 * t < P->L_max && t < 512) t <<= 1;
      P->threads = t;
    }
  }
  const bool shared_path = !P->warp_path && !P->cluster_path;
  // prefer prefetched gathers (unless a synchronous gather mode is requested) and twiddles in
  // shared memory; drop them in that order if they do not fit
  SmemLayout lay = recover_layout(D, P->L_max, pr.k_cap, 1 << hb, true, want_pf);
  if (shared_path) {
    P->tw_smem = true;
    P->prefetch = want_pf;
  }
  if (lay.total + static_reserve > (size_t)optin) {
    lay = recover_layout(D, P->L_max, pr.k_cap, 1 << hb, true, false);
    if (shared_path) P->prefetch = false;
  }
  if (lay.total + static_reserve > (size_t)optin) {
    lay = recover_layout(D, P->L_max, pr.k_cap, 1 << hb, false, false);
    if (shared_path) P->tw_smem = false;
  }
  if (shared_path && lay.total + static_reserve > (size_t)optin) {
    // lines or set too large for shared memory: keep them in a per-CTA slice of global workspace
    P->gm_path = true;
    P->tw_smem = false;
    P->prefetch = false;
    lay = recover_layout(D, P->L_max, pr.k_cap, 1 << hb, false, false);
    P->gm_stride = (lay.total + 255) & ~size_t(255);
  }
  if (shared_path) {
    P->smem = P->gm_path ? 0 : lay.total;
    if (pr.threads > 0) {
      P->threads = pr.threads;
    } else {
      // one CTA per signal: up to 512 threads, 1024 when there are fewer signals than SMs
      const int cap = batch < sms ? 1024 : 512;
      int t = 64;
      while (t < P->L_max && t < cap) t <<= 1;
      P->threads = t;
    }
  }

  // device workspace
  auto cleanup_fail = [&](const char* what, cudaError_t e) {
    free_plan_memory(P);
    delete P;
    return fail(e == cudaErrorMemoryAllocation ? FPSSFT_ERR_ALLOC : FPSSFT_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  const size_t nb = std::max(1, batch);
  if ((e = cudaMalloc(&P->d_shapes, std::max<size_t>(1, P->shapes.size()) * sizeof(Shape))) != cudaSuccess) return cleanup_fail("cudaMalloc shapes", e);
  if ((e = cudaMalloc(&P->d_sig_shape, nb * sizeof(int))) != cudaSuccess) return cleanup_fail("cudaMalloc sig_shape", e);
  if ((e = cudaMalloc(&P->d_sig_T, nb * sizeof(int))) != cudaSuccess) return cleanup_fail("cudaMalloc sig_T", e);
  if ((e = cudaMalloc(&P->d_order, nb * sizeof(int))) != cudaSuccess) return cleanup_fail("cudaMalloc order", e);
  if ((e = cudaMalloc(&P->d_twiddles, std::max<size_t>(1, tw_pool.size()) * sizeof(float2))) != cudaSuccess) return cleanup_fail("cudaMalloc twiddles", e);
  if ((e = cudaMalloc(&P->d_counter, sizeof(int))) != cudaSuccess) return cleanup_fail("cudaMalloc counter", e);
  if (batch > 0) {
    if ((e = cudaMemcpy(P->d_shapes, P->shapes.data(), P->shapes.size() * sizeof(Shape), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail("upload shapes", e);
    if ((e = cudaMemcpy(P->d_sig_shape, P->sig_shape.data(), batch * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail("upload sig_shape", e);
    if ((e = cudaMemcpy(P->d_sig_T, P->sig_T.data(), batch * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail("upload sig_T", e);
    if ((e = cudaMemcpy(P->d_order, P->order.data(), batch * sizeof(int), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail("upload order", e);
    if ((e = cudaMemcpy(P->d_twiddles, tw_pool.data(), tw_pool.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail("upload twiddles", e);
  }

  // kernel attributes and the persistent grid
  fpssft_status st = dispatch_D(D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    if (P->gm_path) P->threads = std::min(P->threads, 512);
    const void* kfn = P->warp_path ? (P->prefetch ? (const void*)k_recover_w<DD, true> : (const void*)k_recover_w<DD, false>)
                    : P->cluster_path ? (P->cluster_gs ? (P->threads > 512 ? (const void*)k_recover_c<DD, 1024, true> : (const void*)k_recover_c<DD, 512, true>)
                                                        : (P->threads > 512 ? (const void*)k_recover_c<DD, 1024, false> : (const void*)k_recover_c<DD, 512, false>))
                    : P->gm_path ? (const void*)k_recover<DD, 512, true>
                    : (P->threads > 512 ? (const void*)k_recover<DD, 1024> : (const void*)k_recover<DD, 512>);
    cudaError_t e2 = ensure_dynamic_smem(kfn, P->smem);
    if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("cudaFuncSetAttribute(recovery kernel): ") + cudaGetErrorString(e2));
    if (P->cluster_path) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = DD + 1;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)(batch * (DD + 1)));
      cfg.blockDim = dim3((unsigned)P->threads);
      cfg.dynamicSmemBytes = P->smem;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int clusters = 0;
      e2 = cudaOccupancyMaxActiveClusters(&clusters, kfn, &cfg);
      if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("cluster occupancy query: ") + cudaGetErrorString(e2));
      if (clusters < 1) return fail(FPSSFT_ERR_UNSUPPORTED, "a cluster of D+1 recovery CTAs cannot be resident with this CTA size / shared memory");
    }
    int per_sm = 0;
    e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, P->threads, P->smem);
    if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("occupancy query: ") + cudaGetErrorString(e2));
    if (per_sm < 1) return fail(FPSSFT_ERR_UNSUPPORTED, "recovery kernel cannot be resident with this CTA size / shared memory");
    if (P->p.ctas_per_sm > 0) per_sm = std::min(per_sm, P->p.ctas_per_sm);
    P->grid = std::max(1, std::min(batch, per_sm * P->sm_count));
    if (P->cluster_path) P->grid = batch * (DD + 1);   // one cluster per signal, not persistent
    if (P->cluster_gs) {   // one slice of global workspace per signal
      const cudaError_t ea = cudaMalloc(&P->d_gm_ws, (size_t)batch * P->gm_stride);
      if (ea != cudaSuccess) return fail(FPSSFT_ERR_ALLOC, std::string("workspace for the cluster path's sets: ") + cudaGetErrorString(ea));
    }
    if (P->gm_path) {   // cap the persistent grid: every CTA owns a workspace slice
      P->grid = std::max(1, std::min(batch, 2 * P->sm_count));
      const size_t bytes = (size_t)P->grid * P->gm_stride;
      const cudaError_t ea = cudaMalloc(&P->d_gm_ws, bytes);
      if (ea != cudaSuccess) return fail(FPSSFT_ERR_ALLOC, std::string("workspace for long lines: ") + cudaGetErrorString(ea));
    }
    const size_t ls = line_smem(DD, P->L_max);
    P->lines_in_smem = ls + sizeof(Shape) + 256 <= (size_t)optin;
    if (P->lines_in_smem) {
      e2 = ensure_dynamic_smem((const void*)k_project<DD>, ls);
      if (e2 == cudaSuccess) e2 = ensure_dynamic_smem((const void*)k_adjoint_project<DD>, ls);
      if (e2 == cudaSuccess) e2 = ensure_dynamic_smem((const void*)k_synth<DD>, ls / 2);
    }
    const size_t ds = (size_t)P->p.k_cap * (sizeof(float2) + (DD + 1) * sizeof(int)) + (size_t)2 * (1 << P->hash_bits) * sizeof(int);
    P->set_in_smem = ds + sizeof(Shape) + 256 <= (size_t)optin;
    if (e2 == cudaSuccess && P->set_in_smem) e2 = ensure_dynamic_smem((const void*)k_decode<DD>, ds);
    if (e2 == cudaSuccess && P->set_in_smem) e2 = ensure_dynamic_smem((const void*)k_finalize<DD>, ds);
    if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("cudaFuncSetAttribute: ") + cudaGetErrorString(e2));
    return FPSSFT_OK;
  });
  if (st != FPSSFT_OK) {
    const std::string msg = g_last_error;
    free_plan_memory(P);
    delete P;
    return fail(st, msg);
  }
  *out = P;
  return FPSSFT_OK;
}

extern "C" fpssft_status fpssft_plan(fpssft_plan_t* out, int D, int batch, const int64_t* dims,
                                     const fpssft_params* params) {
  return fpssft_plan_create(out, D, batch, dims, params);
}

extern "C" void fpssft_plan_destroy(fpssft_plan_t plan) {
  if (!plan) return;
  free_plan_memory(plan);
  delete plan;
}

extern "C" fpssft_status fpssft_plan_get_info(fpssft_plan_t P, fpssft_plan_info* info) {
  if (!P || !info) return fail(FPSSFT_ERR_INVALID, "null plan or info");
  info->D = P->D;
  info->batch = P->batch;
  info->L_max = P->L_max;
  info->T_max = P->T_max;
  info->k_cap = P->p.k_cap;
  info->hash_cap = 1 << P->hash_bits;
  info->n_shapes = P->n_shapes;
  info->threads = P->threads;
  info->grid = P->grid;
  info->smem_bytes = (int)P->smem;
  info->twiddles_in_smem = P->tw_smem ? 1 : 0;
  info->prefetch = P->prefetch ? 1 : 0;
  info->fft_path = P->cluster_path ? 3 : P->warp_path ? 2 : 1;
  info->global_workspace = (P->gm_path || P->cluster_gs) ? 1 : 0;
  return FPSSFT_OK;
}

extern "C" fpssft_status fpssft_plan_get_lengths(fpssft_plan_t P, int32_t* L_out, int32_t* T_out) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  for (int b = 0; b < P->batch; ++b) {
    if (L_out) L_out[b] = P->sig_L[b];
    if (T_out) T_out[b] = P->sig_T[b];
  }
  return FPSSFT_OK;
}

// ================================================================================================
// Host side: launches
// ================================================================================================

static int unit_grid(const fpssft_plan_s* P, long long units, int per_sm) {
  const long long cap = (long long)P->sm_count * per_sm;
  return (int)std::max(1LL, std::min(units, cap));
}

static fpssft_status launch_project(fpssft_plan_t P, const void* cubes, const int64_t* offsets,
                                    const int32_t* alpha, const int32_t* tau, int n_sched, void* out,
                                    void* stream, int dft) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (n_sched < 0) return fail(FPSSFT_ERR_INVALID, "n_sched must be >= 0");
  if (P->batch == 0 || n_sched == 0) return FPSSFT_OK;
  if (!cubes || !offsets || !alpha || !tau || !out) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  if (!P->lines_in_smem) return fail(FPSSFT_ERR_UNSUPPORTED, "lines of this plan exceed one CTA's shared memory");
  ProjectArgs A;
  A.cubes = static_cast<const float2*>(cubes);
  A.offsets = offsets;
  A.alpha = alpha;
  A.tau = tau;
  A.n_sched = n_sched;
  A.tab = P->tables();
  A.batch = P->batch;
  A.L_max = P->L_max;
  A.dft = dft;
  A.out = static_cast<float2*>(out);
  const int grid = unit_grid(P, (long long)P->batch * n_sched, 8);
  const size_t sm = line_smem(P->D, P->L_max);
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    k_project<DD><<<grid, 256, sm, static_cast<cudaStream_t>(stream)>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

extern "C" fpssft_status fpssft_project(fpssft_plan_t P, const void* cubes, const int64_t* offsets,
                                        const int32_t* alpha, const int32_t* tau, int n_sched, void* bins,
                                        void* stream) {
  return launch_project(P, cubes, offsets, alpha, tau, n_sched, bins, stream, 1);
}

extern "C" fpssft_status fpssft_lines(fpssft_plan_t P, const void* cubes, const int64_t* offsets,
                                      const int32_t* alpha, const int32_t* tau, int n_sched, void* lines,
                                      void* stream) {
  return launch_project(P, cubes, offsets, alpha, tau, n_sched, lines, stream, 0);
}

extern "C" fpssft_status fpssft_recover(fpssft_plan_t P, const void* cubes, const int64_t* offsets,
                                        const int32_t* alpha, const int32_t* tau, const int32_t* init_count,
                                        int32_t* out_k, void* out_a, int32_t* out_count, int32_t* out_iters,
                                        int32_t* out_status, void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (P->batch == 0) return FPSSFT_OK;
  if (!cubes || !offsets || !alpha || !tau || !out_k || !out_a || !out_count || !out_iters || !out_status)
    return fail(FPSSFT_ERR_INVALID, "null device pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  RecoverArgs A;
  A.cubes = static_cast<const float2*>(cubes);
  A.offsets = offsets;
  A.alpha = alpha;
  A.tau = tau;
  A.sched_stride = P->T_max * P->D;
  A.tab = P->tables();
  A.work_counter = P->d_counter;
  A.batch = P->batch;
  A.k_cap = P->p.k_cap;
  A.hash_bits = P->hash_bits;
  A.L_max = P->L_max;
  A.tw_smem = P->tw_smem ? 1 : 0;
  A.prefetch = P->prefetch ? 1 : 0;
  A.gather_mode = P->p.gather_mode;
  A.early_stop = P->p.early_stop;
  A.gm_ws = P->d_gm_ws;
  A.gm_stride = P->gm_stride;
  A.th = P->thresholds();
  A.init_count = init_count;
  A.out_k = out_k;
  A.out_a = static_cast<float2*>(out_a);
  A.out_count = out_count;
  A.out_iters = out_iters;
  A.out_status = out_status;
  FPSSFT_CUDA_TRY(cudaMemsetAsync(P->d_counter, 0, sizeof(int), s));
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    if (P->warp_path) {
      if (P->prefetch)
        k_recover_w<DD, true><<<P->grid, P->threads, P->smem, s>>>(A);
      else
        k_recover_w<DD, false><<<P->grid, P->threads, P->smem, s>>>(A);
    } else if (P->cluster_path) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = DD + 1;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3((unsigned)P->grid);
      cfg.blockDim = dim3((unsigned)P->threads);
      cfg.dynamicSmemBytes = P->smem;
      cfg.stream = s;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (P->cluster_gs && P->threads > 512)
        FPSSFT_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_recover_c<DD, 1024, true>, A));
      else if (P->cluster_gs)
        FPSSFT_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_recover_c<DD, 512, true>, A));
      else if (P->threads > 512)
        FPSSFT_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_recover_c<DD, 1024, false>, A));
      else
        FPSSFT_CUDA_TRY(cudaLaunchKernelEx(&cfg, k_recover_c<DD, 512, false>, A));
    } else if (P->gm_path) {
      k_recover<DD, 512, true><<<P->grid, P->threads, 0, s>>>(A);
    } else if (P->threads > 512) {
      k_recover<DD, 1024><<<P->grid, P->threads, P->smem, s>>>(A);
    } else {
      k_recover<DD, 512><<<P->grid, P->threads, P->smem, s>>>(A);
    }
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

extern "C" fpssft_status fpssft_recover_host(fpssft_plan_t P, const void* cubes, const int64_t* offsets,
                                             const int32_t* alpha, const int32_t* tau, const int32_t* init_count,
                                             int32_t* out_k, void* out_a, int32_t* out_count, int32_t* out_iters,
                                             int32_t* out_status, void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (P->batch == 0) return FPSSFT_OK;
  if (!cubes || !offsets || !alpha || !tau || !out_k || !out_a || !out_count || !out_iters || !out_status)
    return fail(FPSSFT_ERR_INVALID, "null host pointer");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t B = (size_t)P->batch, D = (size_t)P->D, kc = (size_t)P->p.k_cap;
  size_t elems = 0;
  for (size_t b = 0; b < B; ++b) {
    if (offsets[b] < 0) return fail(FPSSFT_ERR_INVALID, "negative offset");
    elems = std::max(elems, (size_t)offsets[b] + (size_t)P->shapes[P->sig_shape[b]].N);
  }
  const size_t sched = B * (size_t)P->T_max * D;
  auto alloc = [&](void** ptr, size_t bytes) { return cudaMalloc(ptr, std::max<size_t>(bytes, 16)); };
  if (P->st_cubes != nullptr && elems > P->st_cubes_elems) {
    cudaFree(P->st_cubes);
    P->st_cubes = nullptr;
    P->st_cubes_elems = 0;
    if (alloc(&P->st_cubes, elems * sizeof(float2)) != cudaSuccess) return fail(FPSSFT_ERR_ALLOC, "staging allocation failed");
    P->st_cubes_elems = elems;
  }
  if (P->st_offsets == nullptr) {
    cudaError_t e = cudaSuccess;
    if (P->st_cubes == nullptr) {
      e = alloc(&P->st_cubes, std::max(elems, P->total_elems) * sizeof(float2));
      P->st_cubes_elems = std::max(elems, P->total_elems);
    }
    if (e == cudaSuccess) e = alloc((void**)&P->st_offsets, B * sizeof(int64_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_alpha, sched * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_tau, sched * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_init, B * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_k, B * kc * D * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc(&P->st_a, B * kc * sizeof(float2));
    if (e == cudaSuccess) e = alloc((void**)&P->st_count, B * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_iters, B * sizeof(int32_t));
    if (e == cudaSuccess) e = alloc((void**)&P->st_status, B * sizeof(int32_t));
    if (e != cudaSuccess) return fail(FPSSFT_ERR_ALLOC, std::string("staging allocation: ") + cudaGetErrorString(e));
  }
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_cubes, cubes, elems * sizeof(float2), cudaMemcpyHostToDevice, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_offsets, offsets, B * sizeof(int64_t), cudaMemcpyHostToDevice, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_alpha, alpha, sched * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_tau, tau, sched * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  const int32_t* dinit = nullptr;
  if (init_count) {
    FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_init, init_count, B * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_k, out_k, B * kc * D * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    FPSSFT_CUDA_TRY(cudaMemcpyAsync(P->st_a, out_a, B * kc * sizeof(float2), cudaMemcpyHostToDevice, s));
    dinit = P->st_init;
  }
  fpssft_status st = fpssft_recover(P, P->st_cubes, P->st_offsets, P->st_alpha, P->st_tau, dinit, P->st_k, P->st_a,
                                    P->st_count, P->st_iters, P->st_status, stream);
  if (st != FPSSFT_OK) return st;
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(out_k, P->st_k, B * kc * D * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(out_a, P->st_a, B * kc * sizeof(float2), cudaMemcpyDeviceToHost, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(out_count, P->st_count, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(out_iters, P->st_iters, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(out_status, P->st_status, B * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  FPSSFT_CUDA_TRY(cudaStreamSynchronize(s));
  return FPSSFT_OK;
}

extern "C" fpssft_status fpssft_synth(fpssft_plan_t P, const int32_t* alpha, const int32_t* tau, int n_sched,
                                      const int32_t* k, const void* a, const int32_t* count, int accumulate,
                                      void* bins, void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (n_sched < 0 || accumulate < -1 || accumulate > 1) return fail(FPSSFT_ERR_INVALID, "bad n_sched or accumulate");
  if (P->batch == 0 || n_sched == 0) return FPSSFT_OK;
  if (!alpha || !tau || !k || !a || !count || !bins) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  if (!P->lines_in_smem) return fail(FPSSFT_ERR_UNSUPPORTED, "lines of this plan exceed one CTA's shared memory");
  SynthArgs A;
  A.alpha = alpha;
  A.tau = tau;
  A.n_sched = n_sched;
  A.tab = P->tables();
  A.batch = P->batch;
  A.L_max = P->L_max;
  A.k_cap = P->p.k_cap;
  A.k = k;
  A.a = static_cast<const float2*>(a);
  A.count = count;
  A.accumulate = accumulate;
  A.bins = static_cast<float2*>(bins);
  const int grid = unit_grid(P, (long long)P->batch * n_sched, 8);
  const size_t sm = line_smem(P->D, P->L_max) / 2;
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    k_synth<DD><<<grid, 256, sm, static_cast<cudaStream_t>(stream)>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

extern "C" fpssft_status fpssft_decode(fpssft_plan_t P, const void* bins, const int32_t* alpha, const int32_t* tau,
                                       int32_t* k, void* a, int32_t* count, int32_t* t0_count, int32_t* status,
                                       void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (P->batch == 0) return FPSSFT_OK;
  if (!bins || !alpha || !tau || !k || !a || !count || !t0_count || !status) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  if (!P->set_in_smem) return fail(FPSSFT_ERR_UNSUPPORTED, "fpssft_decode keeps one signal's set in one CTA's shared memory: k_cap too large");
  DecodeArgs A;
  A.bins = static_cast<const float2*>(bins);
  A.alpha = alpha;
  A.tau = tau;
  A.tab = P->tables();
  A.batch = P->batch;
  A.L_max = P->L_max;
  A.k_cap = P->p.k_cap;
  A.hash_bits = P->hash_bits;
  A.th = P->thresholds();
  A.k = k;
  A.a = static_cast<float2*>(a);
  A.count = count;
  A.t0_count = t0_count;
  A.status = status;
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    const size_t ds = (size_t)P->p.k_cap * (sizeof(float2) + (DD + 1) * sizeof(int)) + (size_t)2 * (1 << P->hash_bits) * sizeof(int);
    k_decode<DD><<<unit_grid(P, P->batch, 8), 256, ds, static_cast<cudaStream_t>(stream)>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

extern "C" fpssft_status fpssft_finalize(fpssft_plan_t P, int32_t* k, void* a, int32_t* count, void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (P->batch == 0) return FPSSFT_OK;
  if (!k || !a || !count) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  if (!P->set_in_smem) return fail(FPSSFT_ERR_UNSUPPORTED, "fpssft_finalize keeps one signal's set in one CTA's shared memory: k_cap too large");
  FinalizeArgs A;
  A.tab = P->tables();
  A.batch = P->batch;
  A.k_cap = P->p.k_cap;
  A.sort_cap = 1 << P->hash_bits;
  A.th = P->thresholds();
  A.k = k;
  A.a = static_cast<float2*>(a);
  A.count = count;
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    const size_t ds = (size_t)P->p.k_cap * (sizeof(float2) + (DD + 1) * sizeof(int)) + (size_t)2 * (1 << P->hash_bits) * sizeof(int);
    k_finalize<DD><<<unit_grid(P, P->batch, 8), 256, ds, static_cast<cudaStream_t>(stream)>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

extern "C" fpssft_status fpssft_adjoint(fpssft_plan_t P, fpssft_adj_mode mode, const void* grad_bins,
                                        const int64_t* offsets, const int32_t* alpha, const int32_t* tau, int n_sched,
                                        const int32_t* k, const int32_t* count, void* grad_out, void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (n_sched < 0) return fail(FPSSFT_ERR_INVALID, "n_sched must be >= 0");
  if (mode != FPSSFT_ADJ_PROJECT && mode != FPSSFT_ADJ_SYNTH) return fail(FPSSFT_ERR_INVALID, "unknown adjoint mode");
  if (P->batch == 0) return FPSSFT_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (mode == FPSSFT_ADJ_PROJECT) {
    if (n_sched == 0) return FPSSFT_OK;
    if (!grad_bins || !offsets || !alpha || !tau || !grad_out) return fail(FPSSFT_ERR_INVALID, "null device pointer");
    if (!P->lines_in_smem) return fail(FPSSFT_ERR_UNSUPPORTED, "lines of this plan exceed one CTA's shared memory");
    AdjProjectArgs A;
    A.g = static_cast<const float2*>(grad_bins);
    A.offsets = offsets;
    A.alpha = alpha;
    A.tau = tau;
    A.n_sched = n_sched;
    A.tab = P->tables();
    A.batch = P->batch;
    A.L_max = P->L_max;
    A.grad = static_cast<float2*>(grad_out);
    const int grid = unit_grid(P, (long long)P->batch * n_sched, 8);
    const size_t sm = line_smem(P->D, P->L_max);
    return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
      constexpr int DD = decltype(Dc)::value;
      k_adjoint_project<DD><<<grid, 256, sm, s>>>(A);
      FPSSFT_CUDA_TRY(cudaGetLastError());
      return FPSSFT_OK;
    });
  }
  if (!grad_bins || !alpha || !tau || !k || !count || !grad_out) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  AdjSynthArgs A;
  A.g = static_cast<const float2*>(grad_bins);
  A.alpha = alpha;
  A.tau = tau;
  A.n_sched = n_sched;
  A.tab = P->tables();
  A.batch = P->batch;
  A.L_max = P->L_max;
  A.k_cap = P->p.k_cap;
  A.k = k;
  A.count = count;
  A.grad_a = static_cast<float2*>(grad_out);
  const long long total = (long long)P->batch * P->p.k_cap;
  const int grid = (int)std::max(1LL, std::min((total + 255) / 256, (long long)P->sm_count * 16));
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    k_adjoint_synth<DD><<<grid, 256, 0, s>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}

// ---- random-gather ceiling ------------------------------------------------------------------
// Every thread reads `reads` 8-byte elements at pseudo-random positions of a buffer of n = 2^k
// elements (much larger than L2), optionally together with the next element (the adjacent pair
// the line gather reads for line 0 and line D), and folds them into one output element so the
// loads cannot be dropped.  Positions come from a 64-bit mixing function of (thread, read).
template <int LM, int PAIR>
__global__ void __launch_bounds__(256) k_probe_gather(const float2* __restrict__ buf, unsigned long long mask,
                                                      int reads, unsigned long long seed, float2* out) {
  const unsigned long long tid = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  float ax = 0.f, ay = 0.f;
  unsigned long long h = (tid + 1) * 0x9E3779B97F4A7C15ull ^ seed;
#pragma unroll 8
  for (int r = 0; r < reads; ++r) {
    h += 0x9E3779B97F4A7C15ull;
    unsigned long long z = h;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const unsigned long long i = z & mask;
    const float2 v = load_sample<LM>(buf + i);
    ax += v.x;
    ay += v.y;
    if (PAIR) {
      const float2 w = load_sample<LM>(buf + ((i + 1) & mask));
      ax += w.x;
      ay += w.y;
    }
  }
  out[tid] = make_float2(ax, ay);
}

extern "C" fpssft_status fpssft_probe_gather(const void* buf, int64_t n_elems, int reads_per_thread, int threads_total,
                                             int load_mode, int pair, void* out, void* stream) {
  if (!buf || !out) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  if (n_elems < 2 || (n_elems & (n_elems - 1)) != 0) return fail(FPSSFT_ERR_INVALID, "n_elems must be a power of two >= 2");
  if (reads_per_thread < 1 || threads_total < 256 || threads_total % 256 != 0) return fail(FPSSFT_ERR_INVALID, "bad sizes");
  if (load_mode < 0 || load_mode > 1 || pair < 0 || pair > 1) return fail(FPSSFT_ERR_INVALID, "bad mode");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const unsigned long long mask = (unsigned long long)n_elems - 1;
  const float2* b = static_cast<const float2*>(buf);
  float2* o = static_cast<float2*>(out);
  const int grid = threads_total / 256;
  const unsigned long long seed = 0x2545F4914F6CDD1Dull;
  if (load_mode == 0 && pair == 0) k_probe_gather<0, 0><<<grid, 256, 0, s>>>(b, mask, reads_per_thread, seed, o);
  if (load_mode == 0 && pair == 1) k_probe_gather<0, 1><<<grid, 256, 0, s>>>(b, mask, reads_per_thread, seed, o);
  if (load_mode == 1 && pair == 0) k_probe_gather<1, 0><<<grid, 256, 0, s>>>(b, mask, reads_per_thread, seed, o);
  if (load_mode == 1 && pair == 1) k_probe_gather<1, 1><<<grid, 256, 0, s>>>(b, mask, reads_per_thread, seed, o);
  FPSSFT_CUDA_TRY(cudaGetLastError());
  return FPSSFT_OK;
}

extern "C" fpssft_status fpssft_l2_fetch_granularity(int bytes, int* previous) {
  size_t cur = 0;
  FPSSFT_CUDA_TRY(cudaDeviceGetLimit(&cur, cudaLimitMaxL2FetchGranularity));
  if (previous) *previous = (int)cur;
  if (bytes < 0) return FPSSFT_OK;
  if (bytes != 0 && bytes != 32 && bytes != 64 && bytes != 128) return fail(FPSSFT_ERR_INVALID, "bytes must be 0, 32, 64 or 128");
  FPSSFT_CUDA_TRY(cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, (size_t)bytes));
  return FPSSFT_OK;
}

extern "C" const char* fpssft_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* fpssft_version(void) { return "fpssft-gb300 0.1 (sm_103a)"; }

// ================================================================================================
// Recovery without any device allocation
// ================================================================================================
// Some callers cannot allocate device memory at the time they recover: code running under a
// memory pool or arena owned by someone else, inside a region where cudaMalloc is forbidden or
// would synchronise, or with a fixed device-memory budget.  fpssft_recover_noalloc serves them:
// the plan's tables (shapes, per-signal budgets, work order, twiddles) and the work counter live in
// one file-scope device array of fixed size instead of plan-owned allocations.

namespace {

constexpr size_t kNoallocScratchBytes = (size_t)FPSSFT_NOALLOC_SCRATCH_BYTES;
constexpr int kNoallocMaxShapes = 64;
constexpr int kNoallocMaxDevices = 64;

// The device copy of the tables.  Every GPU that loads the library holds these bytes until the
// process exits.  In host code the name is only a stand-in: kernels receive the device address
// obtained by cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// Host-side staging of the tables (static: building them allocates nothing).
alignas(256) unsigned char g_noalloc_host[kNoallocScratchBytes];
std::mutex g_noalloc_mutex;
unsigned char* g_noalloc_dev[kNoallocMaxDevices] = {};

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

int factorize_into(int L, int* out) {
  int n = L, k = 0;
  const int small[] = {8, 4, 2, 3, 5};
  for (int f : small)
    while (n % f == 0 && k < kMaxStages) { out[k++] = f; n /= f; }
  for (int f = 7; (long long)f * f <= n && k < kMaxStages; f += 2)
    while (n % f == 0 && k < kMaxStages) { out[k++] = f; n /= f; }
  if (n > 1) {
    if (k >= kMaxStages) return -1;
    out[k++] = n;
  }
  return k;
}

}  // namespace

extern "C" fpssft_status fpssft_recover_noalloc(int D, int batch, const int64_t* dims, const fpssft_params* params,
                                                const void* cubes, const int64_t* offsets, const int32_t* alpha,
                                                const int32_t* tau, const int32_t* init_count, int32_t* out_k,
                                                void* out_a, int32_t* out_count, int32_t* out_iters,
                                                int32_t* out_status, void* stream) {
  if (params == nullptr) return fail(FPSSFT_ERR_INVALID, "null params");
  if (D < 1 || D > kMaxD) return fail(FPSSFT_ERR_INVALID, "D must be in [1, 4]");
  if (batch < 0) return fail(FPSSFT_ERR_INVALID, "batch must be >= 0");
  if (batch == 0) return FPSSFT_OK;
  if (!dims || !cubes || !offsets || !alpha || !tau || !out_k || !out_a || !out_count || !out_iters || !out_status)
    return fail(FPSSFT_ERR_INVALID, "null pointer");
  const fpssft_params& pr = *params;
  if (pr.k_cap < 1 || pr.k_cap > (1 << 22)) return fail(FPSSFT_ERR_INVALID, "k_cap must be in [1, 2^22]");
  if (pr.T < 0) return fail(FPSSFT_ERR_INVALID, "T must be >= 0");
  if (!(pr.theta0 >= 0.f) || !(pr.rho >= 0.f) || !(pr.eta >= 0.f)) return fail(FPSSFT_ERR_INVALID, "thresholds must be >= 0");
  if (pr.peel_mode != 0) return fail(FPSSFT_ERR_UNSUPPORTED, "only peel_mode 0 (bins) is implemented on the GPU");
  if (pr.gather_mode < 0 || pr.gather_mode > 3) return fail(FPSSFT_ERR_INVALID, "gather_mode must be in [0, 3]");
  if (pr.threads < 0 || pr.threads > 512 || (pr.threads % 32) != 0) return fail(FPSSFT_ERR_INVALID, "threads must be a multiple of 32 in [0, 512]");

  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  int dev = 0;
  FPSSFT_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoallocMaxDevices) return fail(FPSSFT_ERR_UNSUPPORTED, "device index out of range");
  // set-up, once per device, with that device current: the device address of the scratch array
  if (g_noalloc_dev[dev] == nullptr) {
    void* ptr = nullptr;
    FPSSFT_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
    g_noalloc_dev[dev] = static_cast<unsigned char*>(ptr);
  }
  unsigned char* dscratch = g_noalloc_dev[dev];

  // ---- tables, built in the static host staging area (same rules as fpssft_plan_create) --------
  const size_t off_counter = 0;
  const size_t off_shapes = 256;
  const size_t off_sig_shape = align256(off_shapes + kNoallocMaxShapes * sizeof(Shape));
  const size_t off_sig_T = align256(off_sig_shape + (size_t)batch * sizeof(int));
  const size_t off_order = align256(off_sig_T + (size_t)batch * sizeof(int));
  const size_t off_tw = align256(off_order + (size_t)batch * sizeof(int));
  if (off_tw > kNoallocScratchBytes)
    return fail(FPSSFT_ERR_UNSUPPORTED, "batch exceeds the fixed scratch of fpssft_recover_noalloc (FPSSFT_NOALLOC_SCRATCH_BYTES)");
  Shape* shapes = reinterpret_cast<Shape*>(g_noalloc_host + off_shapes);
  int* sig_shape = reinterpret_cast<int*>(g_noalloc_host + off_sig_shape);
  int* sig_T = reinterpret_cast<int*>(g_noalloc_host + off_sig_T);
  int* order = reinterpret_cast<int*>(g_noalloc_host + off_order);
  float2* tw = reinterpret_cast<float2*>(g_noalloc_host + off_tw);
  const size_t tw_cap = (kNoallocScratchBytes - off_tw) / sizeof(float2);
  int n_shapes = 0, L_max = 1, T_max = 1;
  size_t tw_used = 0;
  for (int b = 0; b < batch; ++b) {
    int dv[kMaxD] = {1, 1, 1, 1};
    long long N = 1, L = 1, nmax = 1;
    for (int d = 0; d < D; ++d) {
      const int64_t n = dims[(size_t)b * D + d];
      if (n < 1 || n > (1 << 24)) return fail(FPSSFT_ERR_INVALID, "every dimension must be in [1, 2^24]");
      dv[d] = (int)n;
      N *= n;
      L = L / std::gcd(L, (long long)n) * n;
      nmax = std::max(nmax, (long long)n);
      if (N > (1LL << 31) - 1 || L > (1LL << 24)) return fail(FPSSFT_ERR_UNSUPPORTED, "cube or line too large (N < 2^31, L <= 2^24)");
    }
    if ((long long)D * L * nmax >= (1LL << 31)) return fail(FPSSFT_ERR_UNSUPPORTED, "D * L * max N_d must stay below 2^31");
    int si = -1;
    for (int q = 0; q < n_shapes && si < 0; ++q) {
      bool same = true;
      for (int d = 0; d < D; ++d) same = same && shapes[q].dims[d] == dv[d];
      if (same) si = q;
    }
    if (si < 0) {
      if (n_shapes >= kNoallocMaxShapes) return fail(FPSSFT_ERR_UNSUPPORTED, "more than 64 distinct shapes in one batch");
      Shape& sh = shapes[n_shapes];
      std::memset(&sh, 0, sizeof(Shape));
      sh.D = D;
      sh.L = (int)L;
      sh.N = (int)N;
      int stride = 1;
      for (int d = D - 1; d >= 0; --d) { sh.dims[d] = dv[d]; sh.strides[d] = stride; stride *= dv[d]; }
      for (int d = 0; d < D; ++d) sh.c[d] = (int)(L / dv[d]);
      const int nst = factorize_into((int)L, sh.radix);
      if (nst < 0) return fail(FPSSFT_ERR_UNSUPPORTED, "too many FFT stages");
      sh.nst = nst;
      for (int d = 0; d < kMaxD; ++d) sh.fdims[d] = make_fastdiv(d < D ? dv[d] : 1);
      sh.fL = make_fastdiv((int)L);
      int ns = 1;
      for (int s = 0; s < nst; ++s) {
        sh.tstep[s] = (int)(L / ((long long)ns * sh.radix[s]));
        sh.fnb[s] = make_fastdiv((int)(L / sh.radix[s]));
        sh.fns[s] = make_fastdiv(ns);
        ns *= sh.radix[s];
      }
      sh.stw_off = -1;  // no per-stage table: the one-CTA-per-signal kernel does not use it
      int reuse = -1;   // twiddle table shared by shapes with the same L
      for (int q = 0; q < n_shapes && reuse < 0; ++q)
        if (shapes[q].L == sh.L) reuse = shapes[q].tw_off;
      if (reuse >= 0) {
        sh.tw_off = reuse;
      } else {
        if (tw_used + (size_t)L > tw_cap)
          return fail(FPSSFT_ERR_UNSUPPORTED, "twiddle tables exceed the fixed scratch of fpssft_recover_noalloc");
        sh.tw_off = (int)tw_used;
        for (long long q = 0; q < L; ++q) {
          const double ang = 2.0 * M_PI * (double)q / (double)L;
          tw[tw_used + q] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        }
        tw_used += (size_t)L;
      }
      si = n_shapes++;
    }
    sig_shape[b] = si;
    const long long budget = std::max(1LL, N / ((long long)(D + 1) * L));
    sig_T[b] = pr.T > 0 ? pr.T : (int)std::min(budget, (long long)1 << 30);
    L_max = std::max(L_max, (int)L);
    T_max = std::max(T_max, sig_T[b]);
    order[b] = b;
  }
  std::sort(order, order + batch, [&](int a, int b) {
    const int La = shapes[sig_shape[a]].L, Lb = shapes[sig_shape[b]].L;
    if (La != Lb) return La > Lb;
    if (sig_T[a] != sig_T[b]) return sig_T[a] > sig_T[b];
    return a < b;
  });
  int hb = 1;
  while ((1 << hb) < 2 * pr.k_cap) ++hb;

  int optin = 0, sms = 1;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (optin <= 0) optin = 227 * 1024;
  if (sms <= 0) sms = 1;
  const size_t static_reserve = sizeof(Shape) + 256;
  const bool want_pf = pr.gather_mode == 3;
  bool tw_smem = true, pf = want_pf;
  SmemLayout lay = recover_layout(D, L_max, pr.k_cap, 1 << hb, true, want_pf);
  if (lay.total + static_reserve > (size_t)optin) { pf = false; lay = recover_layout(D, L_max, pr.k_cap, 1 << hb, true, false); }
  if (lay.total + static_reserve > (size_t)optin) { tw_smem = false; lay = recover_layout(D, L_max, pr.k_cap, 1 << hb, false, false); }
  if (lay.total + static_reserve > (size_t)optin)
    return fail(FPSSFT_ERR_UNSUPPORTED, "lines + recovered set exceed one CTA's shared memory (L_max or k_cap too large)");
  int threads = pr.threads;
  if (threads == 0) {
    threads = 64;
    while (threads < L_max && threads < 512) threads <<= 1;
  }

  // ---- upload the tables and clear the work counter (no allocation: copies into the array) -----
  const size_t bytes = off_tw + tw_used * sizeof(float2);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  FPSSFT_CUDA_TRY(cudaMemcpyAsync(dscratch + off_shapes, g_noalloc_host + off_shapes, bytes - off_shapes,
                                  cudaMemcpyHostToDevice, s));
  FPSSFT_CUDA_TRY(cudaMemsetAsync(dscratch + off_counter, 0, sizeof(int), s));

  RecoverArgs A;
  A.cubes = static_cast<const float2*>(cubes);
  A.offsets = offsets;
  A.alpha = alpha;
  A.tau = tau;
  A.sched_stride = T_max * D;
  A.tab = DeviceTables{reinterpret_cast<const Shape*>(dscratch + off_shapes),
                       reinterpret_cast<const int*>(dscratch + off_sig_shape),
                       reinterpret_cast<const int*>(dscratch + off_sig_T),
                       reinterpret_cast<const int*>(dscratch + off_order),
                       reinterpret_cast<const float2*>(dscratch + off_tw)};
  A.work_counter = reinterpret_cast<int*>(dscratch + off_counter);
  A.batch = batch;
  A.k_cap = pr.k_cap;
  A.hash_bits = hb;
  A.L_max = L_max;
  A.tw_smem = tw_smem ? 1 : 0;
  A.prefetch = pf ? 1 : 0;
  A.gather_mode = pr.gather_mode;
  A.early_stop = pr.early_stop;
  {
    fpssft_plan_s tmp;   // only to reuse the threshold derivation
    tmp.p = pr;
    A.th = tmp.thresholds();
  }
  A.init_count = init_count;
  A.out_k = out_k;
  A.out_a = static_cast<float2*>(out_a);
  A.out_count = out_count;
  A.out_iters = out_iters;
  A.out_status = out_status;
  return dispatch_D(D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    // raise (never lower) the kernel's dynamic shared-memory limit; shared with the plan path
    FPSSFT_CUDA_TRY(ensure_dynamic_smem((const void*)k_recover<DD, 512>, lay.total));
    int per_sm = 0;
    FPSSFT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_recover<DD, 512>, threads, lay.total));
    if (per_sm < 1) return fail(FPSSFT_ERR_UNSUPPORTED, "recovery kernel cannot be resident with this CTA size / shared memory");
    if (pr.ctas_per_sm > 0) per_sm = std::min(per_sm, pr.ctas_per_sm);
    const int grid = std::max(1, std::min(batch, per_sm * sms));
    k_recover<DD, 512><<<grid, threads, lay.total, s>>>(A);
    FPSSFT_CUDA_TRY(cudaGetLastError());
    return FPSSFT_OK;
  });
}
