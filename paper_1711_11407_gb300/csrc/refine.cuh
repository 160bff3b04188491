// Least-squares amplitude refinement on a fixed support, entirely on the device.
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
//
// The decode (Eq. decoding) takes each amplitude from one bin of one line.  Over n_sched schedule
// rows the same amplitudes satisfy y_r = S_r a + noise, where y_r holds the D+1 line DFTs of row r
// (Eq. sample_slice, Eq. hs) and S_r the sparse synthesis of Eq. freqSum.  The refinement solves
//   min_a sum_r ||y_r - S_r a||^2      (per signal)
// by conjugate gradients on the normal equations (S^H S) a = S^H y.  One CG iteration is two
// launches and no host synchronisation:
//   k_refine_normal   per (signal, block of rows): bins = S v (or y - S v) in shared memory, their
//                     squared norm, and g += S^H bins, accumulated over the rows;
//   k_refine_update   per signal: the CG scalars (in FP64) and vector updates.
// Signals whose residual has dropped below tol^2 of its start freeze (step 0), so a fixed number of
// iterations gives the same result as stopping early.
#pragma once

#include "recover_common.cuh"

struct RefineScalars {
  double rr;     // <r, r> of the current residual of the normal equations
  double rr0;    // <r, r> at the start
  double sq;     // accumulated squared norm of the row bins of the last normal pass
  int done;      // converged: later steps leave the signal unchanged
  int pad_;
};

struct RefineNormalArgs {
  const float2* y;          // [batch][n_sched][D+1][L_max] (mode 0 only)
  const int* alpha;
  const int* tau;
  int n_sched;
  DeviceTables tab;
  int batch;
  int L_max;
  int k_cap;
  const int* k;
  const int* count;
  const float2* v;          // [batch][k_cap]: the vector the operator is applied to
  float2* g;                // [batch][k_cap]: += S^H bins (when want_g)
  RefineScalars* sc;        // [batch]: sc.sq += ||bins||^2
  int mode;                 // 0: bins = y - S v; 1: bins = S v
  int want_g;
  int rows_per_unit;
  int units_per_signal;
  int g_in_smem;            // accumulate g over the unit's rows in shared memory, else in global
};

__device__ __forceinline__ double block_sum_double(double v, double* red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x < 32) {
    const int nw = (blockDim.x + 31) >> 5;
    t = (int)threadIdx.x < nw ? red[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

template <int D>
__global__ void __launch_bounds__(256) k_refine_normal(RefineNormalArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Shape sh;
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  __shared__ double s_red[32];
  float2* bins = reinterpret_cast<float2*>(smem);
  float2* gacc = bins + (size_t)(D + 1) * A.L_max;       // [k_cap] when g_in_smem
  int loaded = -1;
  const long long units = (long long)A.batch * A.units_per_signal;
  for (long long u = blockIdx.x; u < units; u += gridDim.x) {
    const int b = (int)(u / A.units_per_signal);
    const int c = (int)(u - (long long)b * A.units_per_signal);
    const int r0 = c * A.rows_per_unit;
    const int r1 = min(A.n_sched, r0 + A.rows_per_unit);
    const int si = A.tab.sig_shape[b];
    __syncthreads();
    if (si != loaded) {
      load_shape(sh, A.tab.shapes, si, nullptr, A.tab.twiddles, false);
      loaded = si;
    }
    const int cnt = min(max(A.count[b], 0), A.k_cap);
    const int* kb = A.k + (size_t)b * A.k_cap * D;
    const float2* vb = A.v + (size_t)b * A.k_cap;
    float2* gb = A.g + (size_t)b * A.k_cap;
    if (A.want_g && A.g_in_smem)
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) gacc[i] = make_float2(0.f, 0.f);
    double sq = 0.0;
    __syncthreads();
    const int L = sh.L;
    const float2* tw = A.tab.twiddles + sh.tw_off;
    for (int r = r0; r < r1; ++r) {
      const long long row = (long long)b * A.n_sched + r;
      if (threadIdx.x < D) {
        const int d = threadIdx.x;
        s_ca[d] = cmodL(sh, d, A.alpha[row * D + d]);
        s_ct[d] = cmodL(sh, d, A.tau[row * D + d]);
      }
      const float2* yr = A.y + row * (D + 1) * (long long)A.L_max;
      for (int i = threadIdx.x; i < (D + 1) * L; i += blockDim.x) {
        const int j = i / L, m = i - j * L;
        bins[i] = A.mode == 0 ? yr[j * A.L_max + m] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const float sign = A.mode == 0 ? -1.f : 1.f;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        int k[D];
#pragma unroll
        for (int d = 0; d < D; ++d) k[d] = kb[i * D + d];
        if (on_grid<D>(sh, k)) project_entry<D>(bins, L, sh, k, vb[i], s_ca, s_ct, tw, sign);
      }
      __syncthreads();
      float sqr = 0.f;   // this thread's few bins of the row in FP32, the sums over rows and threads in FP64
      for (int i = threadIdx.x; i < (D + 1) * L; i += blockDim.x) {
        const float2 q = bins[i];
        sqr = fmaf(q.x, q.x, fmaf(q.y, q.y, sqr));
      }
      sq += (double)sqr;
      if (A.want_g) {
        // g_i += sum_j conj(W^(p + [j > 0] c_{j-1} k_{j-1})) bins_j(m(k_i)); conj(W^q) = tw[q]
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
          int k[D];
#pragma unroll
          for (int d = 0; d < D; ++d) k[d] = kb[i * D + d];
          if (!on_grid<D>(sh, k)) continue;
          int msum = 0, psum = 0;
#pragma unroll
          for (int d = 0; d < D; ++d) {
            msum += s_ca[d] * k[d];
            psum += s_ct[d] * k[d];
          }
          const int m = fmod_(msum, sh.fL);
          const int p = fmod_(psum, sh.fL);
          float2 acc = cmul(tw[p], bins[m]);
#pragma unroll
          for (int d = 0; d < D; ++d) {
            int q = p + sh.c[d] * k[d];
            if (q >= L) q -= L;
            acc = cadd(acc, cmul(tw[q], bins[(d + 1) * L + m]));
          }
          if (A.g_in_smem) {
            gacc[i] = cadd(gacc[i], acc);   // entry i belongs to this thread for every row
          } else {
            atomicAdd(&gb[i].x, acc.x);
            atomicAdd(&gb[i].y, acc.y);
          }
        }
      }
      __syncthreads();
    }
    const double tot = block_sum_double(sq, s_red);
    if (threadIdx.x == 0) atomicAdd(&A.sc[b].sq, tot);
    if (A.want_g && A.g_in_smem) {
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        if (A.units_per_signal == 1) {
          gb[i] = gacc[i];
        } else {
          atomicAdd(&gb[i].x, gacc[i].x);
          atomicAdd(&gb[i].y, gacc[i].y);
        }
      }
    }
  }
}

struct RefineUpdateArgs {
  int batch;
  int k_cap;
  const int* count;
  float2* a;        // [batch][k_cap]
  float2* r;        // residual of the normal equations
  float2* p;        // search direction
  float2* g;        // result of the last normal pass (cleared here)
  RefineScalars* sc;
  float* resid;     // [batch] (mode 2), nullable
  double tol2;
  int mode;         // 0: start (r = p = g); 1: one CG step; 2: residual norm out
};

__global__ void __launch_bounds__(256) k_refine_update(RefineUpdateArgs A) {
  __shared__ double s_red[32];
  __shared__ double s_step, s_beta;
  __shared__ int s_skip;
  for (int b = blockIdx.x; b < A.batch; b += gridDim.x) {
    const int cnt = min(max(A.count[b], 0), A.k_cap);
    const size_t base = (size_t)b * A.k_cap;
    RefineScalars& S = A.sc[b];
    __syncthreads();
    if (A.mode == 2) {
      if (threadIdx.x == 0) {
        if (A.resid) A.resid[b] = (float)sqrt(S.sq);
        S.sq = 0.0;
      }
      continue;
    }
    if (A.mode == 0) {
      double rr = 0.0;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float2 gi = A.g[base + i];
        A.r[base + i] = gi;
        A.p[base + i] = gi;
        A.g[base + i] = make_float2(0.f, 0.f);
        rr += (double)gi.x * gi.x + (double)gi.y * gi.y;
      }
      const double tot = block_sum_double(rr, s_red);
      if (threadIdx.x == 0) {
        S.rr = tot;
        S.rr0 = tot;
        S.sq = 0.0;
        S.done = tot <= 0.0 ? 1 : 0;
      }
      continue;
    }
    if (threadIdx.x == 0) {
      const double qq = S.sq;
      s_skip = S.done || !(qq > 0.0);
      s_step = s_skip ? 0.0 : S.rr / qq;
    }
    __syncthreads();
    const float step = (float)s_step;
    double rr = 0.0;
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
      const float2 gi = A.g[base + i];
      A.g[base + i] = make_float2(0.f, 0.f);
      if (s_skip) continue;
      const float2 pi = A.p[base + i];
      float2 ai = A.a[base + i];
      float2 ri = A.r[base + i];
      ai = make_float2(fmaf(step, pi.x, ai.x), fmaf(step, pi.y, ai.y));
      ri = make_float2(fmaf(-step, gi.x, ri.x), fmaf(-step, gi.y, ri.y));
      A.a[base + i] = ai;
      A.r[base + i] = ri;
      rr += (double)ri.x * ri.x + (double)ri.y * ri.y;
    }
    const double tot = block_sum_double(rr, s_red);
    if (threadIdx.x == 0) {
      if (!s_skip) {
        s_beta = S.rr > 0.0 ? tot / S.rr : 0.0;
        S.rr = tot;
        if (tot <= A.tol2 * S.rr0) S.done = 1;
      } else {
        s_beta = 0.0;
      }
      S.sq = 0.0;
    }
    __syncthreads();
    if (!s_skip) {
      const float beta = (float)s_beta;
      for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float2 ri = A.r[base + i];
        const float2 pi = A.p[base + i];
        A.p[base + i] = make_float2(fmaf(beta, pi.x, ri.x), fmaf(beta, pi.y, ri.y));
      }
    }
  }
}
