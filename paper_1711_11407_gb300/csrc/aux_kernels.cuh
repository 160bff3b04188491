// Kernels of the building-block calls: projection, raw lines, synthesis / peel, the unfused decode
// and finalize steps, and the two adjoints.
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
#pragma once

#include "recover_common.cuh"

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
    const float2* stw = sh.stw_off < 0 ? nullptr : A.tab.twiddles + sh.stw_off;
    const float2* res = A.dft ? fft_lines(bufA, bufB, D + 1, sh, A.tab.twiddles + sh.tw_off, 1.0f / (float)L, stw) : bufA;
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
  int* accepted;    // nullable
  int* status;
};

template <int D>
__global__ void __launch_bounds__(256) k_decode(DecodeArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_count, s_t0, s_ovf, s_acc;
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
      s_acc = 0;
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
                   A.tab.twiddles + sh.tw_off, A.th, &s_t0, &s_ovf, &s_acc);
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
      if (A.accepted) A.accepted[b] = s_acc;
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
    const float2* res = fft_lines(bufA, bufB, D + 1, sh, A.tab.twiddles + sh.tw_off, 1.0f / (float)L,
                                  sh.stw_off < 0 ? nullptr : A.tab.twiddles + sh.stw_off);
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
