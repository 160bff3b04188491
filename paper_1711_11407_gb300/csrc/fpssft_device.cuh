// Device building blocks of the FPS-SFT recovery loop (sm_103a).
//
// Paper: Wang, Patel, Petropulu, "FPS-SFT: A Multi-dimensional Sparse Fourier Transform Based on
// the Fourier Projection-slice Theorem", arXiv 1711.11407.
//
// The building blocks work on the lines and set one CTA holds: the D+1 lines of one iteration in
// shared memory as [D+1][L] complex64 (line-major), or one line (fft_line, the cluster path), the
// recovered set as a dense list plus an open-addressing index (or per-bin buckets, the register
// path), and every phase ends with a CTA barrier issued by the caller.  Integer work (grid points, bins, twiddle indices) is exact; bins are FP32; the
// 1-sparsity tests and the phase decode are evaluated in FP64 from the FP32 bins.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fpssft {

constexpr int kMaxD = 4;
constexpr int kMaxStages = 24;
constexpr int kEmpty = -1;           // empty hash slot (keys are linear indices >= 0)

// Division by a runtime-invariant divisor d >= 1 as a multiply-high and a shift (Granlund and
// Montgomery's round-up method): with l = ceil(log2 d) and m = floor(2^32 (2^l - d) / d) + 1,
// n / d = (umulhi(n, m) + n) >> l for every 0 <= n < 2^31.  The host fills (m, l, d).
struct FastDiv {
  unsigned m;
  int l;
  int d;
  int pad_;
};

__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
  return (int)((__umulhi((unsigned)n, f.m) + (unsigned)n) >> f.l);
}
__device__ __forceinline__ int fmod_(int n, const FastDiv& f) { return n - fdiv(n, f) * f.d; }

// One distinct cube shape of a batch, with its line length and FFT factorisation.
struct Shape {
  int D;
  int L;                     // LCM of the dims (Lemma 1)
  int N;                     // number of grid points
  int nst;                   // FFT stages
  int tw_off;                // offset of the L-entry twiddle table in the pool
  int stw_off;               // offset of the (L-1)-entry per-stage twiddle table (-1: none)
  int dims[kMaxD];
  int strides[kMaxD];        // row-major element strides (last dimension fastest)
  int c[kMaxD];              // L / N_d
  int radix[kMaxStages];     // radices, product = L
  int tstep[kMaxStages];     // L / (Ns R): twiddle stride of each stage
  FastDiv fdims[kMaxD];      // division by N_d
  FastDiv fL;                // division by L
  FastDiv fnb[kMaxStages];   // division by L / R of each stage
  FastDiv fns[kMaxStages];   // division by Ns (product of the earlier radices) of each stage
};

// [c_d v]_L in [0, L) for any int v: v is first reduced into [0, N_d) (schedule entries are never
// trusted to be in range), then c_d v < L N_d < 2^31 (a plan invariant) is reduced by L.
__device__ __forceinline__ int cmodL(const Shape& sh, int d, int v) {
  const int vr = fmod_(v & 0x3fffffff, sh.fdims[d]);
  return fmod_(sh.c[d] * vr, sh.fL);
}

// True when every component lies on the grid (0 <= k_d < N_d); entries that fail are skipped by
// every kernel that reads caller-supplied frequencies.
template <int D>
__device__ __forceinline__ bool on_grid(const Shape& sh, const int* k) {
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) ok = ok && k[d] >= 0 && k[d] < sh.dims[d];
  return ok;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {   // a * conj(b)
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_mj(float2 a) { return make_float2(a.y, -a.x); }   // a * (-j)
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }

// ------------------------------------------------------------------------------------------------
// a1: gather the D+1 lines (Eq. sample_slice; offsets tau and tau + e_d, Sec. 2.3)
// ------------------------------------------------------------------------------------------------
// buf[j * L + l] = x(n_j(l)),  n_d(l) = [alpha_d l + tau_d]_{N_d},  line d+1 adds e_d (mod N_d).
// One thread owns one l and issues the D+1 loads of that l back to back; line D (offset on the
// fastest dimension) is the neighbour of line 0 in memory and usually shares its 32-byte sector.
// Global loads of one sample: LM = 0 through L1 (read-only path, ld.global.nc), LM = 1 cached in
// L2 only (ld.global.cg).
template <int LM>
__device__ __forceinline__ float2 load_sample(const float2* p) {
  if (LM == 1) return __ldcg(p);
  return __ldg(p);
}

template <int D, int LM = 0>
__device__ __forceinline__ void gather_lines(float2* __restrict__ buf, const float2* __restrict__ x,
                                             const Shape& sh, const int* __restrict__ alpha,
                                             const int* __restrict__ tau) {
  const int L = sh.L;
  int al[D], ta[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    al[d] = fmod_(__ldg(alpha + d) & 0x3fffffff, sh.fdims[d]);
    ta[d] = fmod_(__ldg(tau + d) & 0x3fffffff, sh.fdims[d]);
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    int n[D];
    int base = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      n[d] = fmod_(al[d] * l + ta[d], sh.fdims[d]);
      base += n[d] * sh.strides[d];
    }
    float2 v[D + 1];
    v[0] = load_sample<LM>(x + base);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int step = (n[d] + 1 == sh.dims[d]) ? -(sh.dims[d] - 1) * sh.strides[d] : sh.strides[d];
      v[d + 1] = load_sample<LM>(x + base + step);
    }
#pragma unroll
    for (int j = 0; j <= D; ++j) buf[j * L + l] = v[j];
  }
}

// Asynchronous variant (cp.async, 8 bytes per sample, through L1): the copies land in shared
// memory after the issuing thread's cp.async.wait_group and a CTA barrier.  Lets the gather of
// iteration t+1 (whose slope and offset are known in advance) overlap iteration t's compute.
__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

template <int D>
__device__ __forceinline__ void gather_lines_async(float2* __restrict__ buf, const float2* __restrict__ x,
                                                   const Shape& sh, const int* __restrict__ alpha,
                                                   const int* __restrict__ tau) {
  const int L = sh.L;
  int al[D], ta[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    al[d] = fmod_(__ldg(alpha + d) & 0x3fffffff, sh.fdims[d]);
    ta[d] = fmod_(__ldg(tau + d) & 0x3fffffff, sh.fdims[d]);
  }
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    int n[D];
    int base = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      n[d] = fmod_(al[d] * l + ta[d], sh.fdims[d]);
      base += n[d] * sh.strides[d];
    }
    cp_async8(buf + l, x + base);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      const int step = (n[d] + 1 == sh.dims[d]) ? -(sh.dims[d] - 1) * sh.strides[d] : sh.strides[d];
      cp_async8(buf + (d + 1) * L + l, x + base + step);
    }
  }
  cp_async_commit();
}

// Grid-point address of line j at position l (used by the projection adjoint's scatter).
template <int D>
__device__ __forceinline__ int line_address(const Shape& sh, const int* al, const int* ta, int j, int l) {
  int base = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const int nd = fmod_(al[d] * l + ta[d] + (j == d + 1 ? 1 : 0), sh.fdims[d]);
    base += nd * sh.strides[d];
  }
  return base;
}

// Line j alone into buf[0, L) (one CTA per line): synchronous (LM as in load_sample) or, ASYNC,
// as cp.async copies committed as one group.
template <int D, int LM, bool ASYNC>
__device__ __forceinline__ void gather_one_line(float2* __restrict__ buf, const float2* __restrict__ x,
                                                const Shape& sh, const int* __restrict__ alpha,
                                                const int* __restrict__ tau, int j) {
  int al[D], ta[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    al[d] = fmod_(__ldg(alpha + d) & 0x3fffffff, sh.fdims[d]);
    ta[d] = fmod_(__ldg(tau + d) & 0x3fffffff, sh.fdims[d]);
  }
  for (int l = threadIdx.x; l < sh.L; l += blockDim.x) {
    const float2* src = x + line_address<D>(sh, al, ta, j, l);
    if (ASYNC)
      cp_async8(buf + l, src);
    else
      buf[l] = load_sample<LM>(src);
  }
  if (ASYNC) cp_async_commit();
}

// ------------------------------------------------------------------------------------------------
// a2: L-point DFT of every line (Eq. hs), mixed-radix Stockham in shared memory
// ------------------------------------------------------------------------------------------------
// Stage with radix R and span Ns (product of the earlier radices): butterfly j of a line reads
// in[j + i L/R], multiplies input i by w^(i (j mod Ns) L/(Ns R)) with w = exp(-j 2 pi / L), takes the
// R-point DFT and writes out[(j - j mod Ns) R + j mod Ns + i Ns].  After all stages the output is
// in natural order.  tw[q] = exp(-j 2 pi q / L), computed in FP64 on the host and rounded to FP32.
template <int R>
__device__ __forceinline__ void butterfly(float2 (&v)[R]);

template <>
__device__ __forceinline__ void butterfly<2>(float2 (&v)[2]) {
  const float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <>
__device__ __forceinline__ void butterfly<3>(float2 (&v)[3]) {
  const float h = 0.86602540378443865f;  // sin(2 pi / 3)
  const float2 t1 = cadd(v[1], v[2]);
  const float2 t2 = csub(v[1], v[2]);
  const float2 m = make_float2(v[0].x - 0.5f * t1.x, v[0].y - 0.5f * t1.y);
  const float2 n = cscale(mul_mj(t2), h);
  v[0] = cadd(v[0], t1);
  v[1] = cadd(m, n);
  v[2] = csub(m, n);
}

template <>
__device__ __forceinline__ void butterfly<4>(float2 (&v)[4]) {
  const float2 t0 = cadd(v[0], v[2]);
  const float2 t1 = csub(v[0], v[2]);
  const float2 t2 = cadd(v[1], v[3]);
  const float2 t3 = mul_mj(csub(v[1], v[3]));
  v[0] = cadd(t0, t2);
  v[2] = csub(t0, t2);
  v[1] = cadd(t1, t3);
  v[3] = csub(t1, t3);
}

template <>
__device__ __forceinline__ void butterfly<5>(float2 (&v)[5]) {
  const float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;   // cos(2 pi/5), cos(4 pi/5)
  const float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;    // sin(2 pi/5), sin(4 pi/5)
  const float2 t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
  const float2 t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
  const float2 a0 = v[0];
  const float2 b1 = make_float2(a0.x + c1 * t1.x + c2 * t2.x, a0.y + c1 * t1.y + c2 * t2.y);
  const float2 b2 = make_float2(a0.x + c2 * t1.x + c1 * t2.x, a0.y + c2 * t1.y + c1 * t2.y);
  const float2 e1 = mul_mj(make_float2(s1 * t3.x + s2 * t4.x, s1 * t3.y + s2 * t4.y));
  const float2 e2 = mul_mj(make_float2(s2 * t3.x - s1 * t4.x, s2 * t3.y - s1 * t4.y));
  v[0] = cadd(a0, cadd(t1, t2));
  v[1] = cadd(b1, e1);
  v[4] = csub(b1, e1);
  v[2] = cadd(b2, e2);
  v[3] = csub(b2, e2);
}

template <>
__device__ __forceinline__ void butterfly<8>(float2 (&v)[8]) {
  const float c = 0.70710678118654752f;
  float2 e[4] = {v[0], v[2], v[4], v[6]};
  float2 o[4] = {v[1], v[3], v[5], v[7]};
  butterfly<4>(e);
  butterfly<4>(o);
  // o[q] *= exp(-j 2 pi q / 8)
  o[1] = make_float2(c * (o[1].x + o[1].y), c * (o[1].y - o[1].x));
  o[2] = mul_mj(o[2]);
  o[3] = make_float2(c * (o[3].y - o[3].x), -c * (o[3].x + o[3].y));
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    v[q] = cadd(e[q], o[q]);
    v[q + 4] = csub(e[q], o[q]);
  }
}

// stw (may be null): the per-stage twiddle table of fft_line (entry i Ns + k - 1 = tw[i k tstep]),
// read at consecutive addresses by consecutive butterflies instead of the strided tw reads.
template <int R>
__device__ __forceinline__ void fft_stage(const float2* __restrict__ in, float2* __restrict__ out, int L,
                                          int nlines, int Ns, int tstep, const FastDiv& fnb, const FastDiv& fns,
                                          const float2* __restrict__ tw, const float2* __restrict__ stw, float sc) {
  const int nb = fnb.d;
  const int total = nlines * nb;
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int line = fdiv(w, fnb);
    const int j = w - line * nb;
    const float2* src = in + line * L;
    float2* dst = out + line * L;
    const int k = fmod_(j, fns);
    float2 v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) v[i] = src[j + i * nb];
    if (k != 0) {
#pragma unroll
      for (int i = 1; i < R; ++i) v[i] = cmul(v[i], stw ? stw[i * Ns + k - 1] : tw[i * k * tstep]);
    }
    butterfly<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int i = 0; i < R; ++i) dst[base + i * Ns] = cscale(v[i], sc);
  }
}

// Any radix (used for prime factors other than 2, 3, 5): O(R^2) per butterfly, inputs re-read
// from shared memory.  One work item per output (line, butterfly j, output q), so that a stage
// with few butterflies -- a large prime R, or R = L for a prime line length -- still spreads its
// L R multiply-adds over every thread of the CTA.
__device__ __forceinline__ void fft_stage_generic(const float2* __restrict__ in, float2* __restrict__ out,
                                                  int L, int nlines, int Ns, int R, int tstep, const FastDiv& fnb,
                                                  const FastDiv& fns, const float2* __restrict__ tw,
                                                  const float2* __restrict__ stw, float sc) {
  const int nb = fnb.d;
  const int rstep = nb;              // exp(-j 2 pi x / R) = tw[(x mod R) * L / R]
  const int total = nlines * L;      // nlines * nb * R outputs
  for (int w = threadIdx.x; w < total; w += blockDim.x) {
    const int line = w / L;
    const int r = w - line * L;      // r = q nb + j
    const int q = fdiv(r, fnb);
    const int j = r - q * nb;
    const float2* src = in + line * L;
    const int k = fmod_(j, fns);
    float2 acc = make_float2(0.f, 0.f);
    int x = 0;                       // (i q) mod R, advanced incrementally
    for (int i = 0; i < R; ++i) {
      float2 v = src[j + i * nb];
      if (k != 0 && i != 0) v = cmul(v, stw ? stw[i * Ns + k - 1] : tw[i * k * tstep]);
      acc = cadd(acc, cmul(v, tw[x * rstep]));
      x += q;
      if (x >= R) x -= R;
    }
    out[line * L + (j - k) * R + k + q * Ns] = cscale(acc, sc);
  }
}

// Forward DFT (exp(-j ...)) of nlines contiguous lines of length sh.L held in buf0, scaled by
// `scale` at the last stage; buf1 is the ping-pong partner.  Ends with a barrier after each stage
// and returns the buffer holding the result.
__device__ __forceinline__ float2* fft_lines(float2* buf0, float2* buf1, int nlines, const Shape& sh,
                                             const float2* __restrict__ tw, float scale,
                                             const float2* __restrict__ stw = nullptr) {
  float2* in = buf0;
  float2* out = buf1;
  int Ns = 1;
  const int L = sh.L;
  for (int s = 0; s < sh.nst; ++s) {
    const int R = sh.radix[s];
    const int ts = sh.tstep[s];
    const float sc = (s == sh.nst - 1) ? scale : 1.f;
    switch (R) {
      case 2: fft_stage<2>(in, out, L, nlines, Ns, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
      case 3: fft_stage<3>(in, out, L, nlines, Ns, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
      case 4: fft_stage<4>(in, out, L, nlines, Ns, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
      case 5: fft_stage<5>(in, out, L, nlines, Ns, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
      case 8: fft_stage<8>(in, out, L, nlines, Ns, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
      default: fft_stage_generic(in, out, L, nlines, Ns, R, ts, sh.fnb[s], sh.fns[s], tw, stw, sc); break;
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    Ns *= R;
  }
  return in;
}

// One line per CTA (the cluster path), with two changes that remove most shared-memory bank
// conflicts of the stages above:
//  * the intermediate buffers (not the first stage's input, not the last stage's output) keep one
//    float2 of padding after every 16 elements when the stage writing them has radix 2, 4 or 8 and
//    span Ns < 16: the writes out[(j - k) R + k + i Ns] of consecutive butterflies are then spread
//    over distinct banks instead of R/Ns-way conflicts;
//  * the twiddles w^(i k L/(Ns R)) of each stage come from a per-stage table laid out as
//    stw[i Ns + k - 1] (i = 1..R-1, k < Ns; the stages tile [0, L-1) exactly since
//    sum_s (R_s - 1) Ns_s = L - 1), read at consecutive addresses by consecutive butterflies.
// Buffers need padq(L - 1) + 1 elements.
__device__ __forceinline__ int padq(int q) { return q + (q >> 4); }

__device__ __forceinline__ bool stage_pads_output(const Shape& sh, int s, int Ns) {
  const int R = sh.radix[s];
  return s < sh.nst - 1 && (R == 2 || R == 4 || R == 8) && Ns < 16;
}

template <int R>
__device__ __forceinline__ void fft_stage_line(const float2* __restrict__ in, float2* __restrict__ out, int L, int Ns,
                                               const FastDiv& fns, const float2* __restrict__ stw, bool pin, bool pout,
                                               float sc) {
  const int nb = L / R;
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    const int k = fmod_(j, fns);
    float2 v[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int q = j + i * nb;
      v[i] = in[pin ? padq(q) : q];
    }
    if (k != 0) {
#pragma unroll
      for (int i = 1; i < R; ++i) v[i] = cmul(v[i], stw[i * Ns + k - 1]);
    }
    butterfly<R>(v);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int i = 0; i < R; ++i) {
      const int q = base + i * Ns;
      out[pout ? padq(q) : q] = cscale(v[i], sc);
    }
  }
}

__device__ __forceinline__ void fft_stage_line_generic(const float2* __restrict__ in, float2* __restrict__ out, int L,
                                                       int Ns, int R, const FastDiv& fns, const float2* __restrict__ tw,
                                                       const float2* __restrict__ stw, bool pin, bool pout, float sc) {
  const int nb = L / R;
  for (int r = threadIdx.x; r < L; r += blockDim.x) {   // one output (butterfly j, output q) per item
    const int q = r / nb;
    const int j = r - q * nb;
    const int k = fmod_(j, fns);
    float2 acc = make_float2(0.f, 0.f);
    int x = 0;                       // (i q) mod R
    for (int i = 0; i < R; ++i) {
      const int qi = j + i * nb;
      float2 v = in[pin ? padq(qi) : qi];
      if (k != 0 && i != 0) v = cmul(v, stw[i * Ns + k - 1]);
      acc = cadd(acc, cmul(v, tw[x * nb]));   // exp(-j 2 pi x / R) = tw[x L / R]
      x += q;
      if (x >= R) x -= R;
    }
    const int qo = (j - k) * R + k + q * Ns;
    out[pout ? padq(qo) : qo] = cscale(acc, sc);
  }
}

// Forward DFT of one line of length sh.L in buf0 (natural order in, natural order out), scaled by
// `scale`; buf1 is the ping-pong partner.  A barrier ends every stage; returns the result buffer.
__device__ __forceinline__ float2* fft_line(float2* buf0, float2* buf1, const Shape& sh, const float2* __restrict__ tw,
                                            const float2* __restrict__ stw, float scale) {
  float2* in = buf0;
  float2* out = buf1;
  int Ns = 1;
  bool pin = false;
  const int L = sh.L;
  for (int s = 0; s < sh.nst; ++s) {
    const int R = sh.radix[s];
    const float sc = (s == sh.nst - 1) ? scale : 1.f;
    const bool pout = stage_pads_output(sh, s, Ns);
    switch (R) {
      case 2: fft_stage_line<2>(in, out, L, Ns, sh.fns[s], stw, pin, pout, sc); break;
      case 3: fft_stage_line<3>(in, out, L, Ns, sh.fns[s], stw, pin, pout, sc); break;
      case 4: fft_stage_line<4>(in, out, L, Ns, sh.fns[s], stw, pin, pout, sc); break;
      case 5: fft_stage_line<5>(in, out, L, Ns, sh.fns[s], stw, pin, pout, sc); break;
      case 8: fft_stage_line<8>(in, out, L, Ns, sh.fns[s], stw, pin, pout, sc); break;
      default: fft_stage_line_generic(in, out, L, Ns, R, sh.fns[s], tw, stw, pin, pout, sc); break;
    }
    __syncthreads();
    float2* t = in;
    in = out;
    out = t;
    Ns *= R;
    pin = pout;
  }
  return in;
}

// ------------------------------------------------------------------------------------------------
// The recovered set: dense list + open-addressing index (a5)
// ------------------------------------------------------------------------------------------------
struct SetView {
  int* lk;        // [D][k_cap] frequency components
  int* lkey;      // [k_cap] row-major linear index
  float2* la;     // [k_cap] amplitudes
  int* hkey;      // [hash_cap] key or kEmpty
  int* hidx;      // [hash_cap] list position (-1: key claimed by an insert that overflowed)
  int* count;     // entries appended (may exceed k_cap after an overflow; clamp when reading)
  int k_cap;
  int hash_bits;
};

__device__ __forceinline__ unsigned hash_slot(int key, int bits) {
  return ((unsigned)key * 2654435761u) >> (32 - bits);
}

// Insert (k, a) or add a to the existing entry of key.  Within one iteration every key comes from
// at most one bin (the bin of k is unique), so concurrent calls carry distinct keys and an existing
// key was inserted (and fully written) in an earlier iteration.  Returns false on overflow.
template <int D>
__device__ __forceinline__ bool set_insert(const SetView& s, const int* k, int key, float2 a) {
  const unsigned mask = (1u << s.hash_bits) - 1u;
  unsigned h = hash_slot(key, s.hash_bits);
  for (unsigned probe = 0; probe <= mask; ++probe) {
    const int old = atomicCAS(&s.hkey[h], kEmpty, key);
    if (old == kEmpty) {
      const int idx = atomicAdd(s.count, 1);
      if (idx >= s.k_cap) {
        s.hidx[h] = -1;
        return false;
      }
#pragma unroll
      for (int d = 0; d < D; ++d) s.lk[d * s.k_cap + idx] = k[d];
      s.lkey[idx] = key;
      s.la[idx] = a;
      s.hidx[h] = idx;
      return true;
    }
    if (old == key) {
      const int idx = s.hidx[h];
      if (idx < 0 || idx >= s.k_cap) return false;   // overflowed claim (or a repeated resume key)
      s.la[idx] = cadd(s.la[idx], a);
      return true;
    }
    h = (h + 1u) & mask;
  }
  return false;   // unreachable at load factor <= 1/2
}

// ------------------------------------------------------------------------------------------------
// a3: peel -- subtract the recovered set's bins (Eq. freqSum over the set, Sec. 2.2)
// ------------------------------------------------------------------------------------------------
// For entry (k, a): m = [sum_d ca_d k_d]_L with ca_d = [c_d alpha_d]_L; p = [sum_d ct_d k_d]_L with
// ct_d = [c_d tau_d]_L; line 0 gets a W^p and line d+1 gets a W^(p + c_d k_d), W = exp(j 2 pi / L)
// (conj of the forward table).  sign = -1 subtracts (peel), +1 adds (synthesis).
template <int D>
__device__ __forceinline__ void project_entry(float2* bins, int line_stride, const Shape& sh, const int* k,
                                              float2 a, const int* ca, const int* ct,
                                              const float2* __restrict__ tw, float sign) {
  const int L = sh.L;
  int msum = 0, psum = 0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    msum += ca[d] * k[d];
    psum += ct[d] * k[d];
  }
  const int m = fmod_(msum, sh.fL);
  const int p = fmod_(psum, sh.fL);
  float2 v = cmulc(a, tw[p]);
  atomicAdd(&bins[m].x, sign * v.x);
  atomicAdd(&bins[m].y, sign * v.y);
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int q = p + sh.c[d] * k[d];
    if (q >= L) q -= L;
    v = cmulc(a, tw[q]);
    atomicAdd(&bins[(d + 1) * line_stride + m].x, sign * v.x);
    atomicAdd(&bins[(d + 1) * line_stride + m].y, sign * v.y);
  }
}

template <int D>
__device__ __forceinline__ void peel_set(float2* bins, const Shape& sh, const SetView& s, int count,
                                         const int* ca, const int* ct, const float2* __restrict__ tw) {
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    int k[D];
#pragma unroll
    for (int d = 0; d < D; ++d) k[d] = s.lk[d * s.k_cap + i];
    project_entry<D>(bins, sh.L, sh, k, s.la[i], ca, ct, tw, -1.f);
  }
}

// ------------------------------------------------------------------------------------------------
// a4 + a5: 1-sparsity tests, OFDM-trick decode (Eq. decoding) and merge
// ------------------------------------------------------------------------------------------------
// The decisions T0..T2 are defined in FP64 on the FP32 bins.  GB300 runs FP64 at a small
// fraction of its FP32 rate, so every bin is first evaluated in FP32 and the FP32 verdict is used
// only when it is certified: the FP32 value lies outside a guard band around the threshold that is
// wider than the largest possible FP32-vs-FP64 difference (FP32 products and sums: relative error
// <= 2^-23; atan2f: <= 3 ulp by the CUDA math library's documented bound; the band keeps a factor
// >= 4 on top).  Bins inside a band are re-evaluated entirely in FP64, so every verdict equals the
// one a pure FP64 evaluation gives.  fp64_all = 1 forces the FP64 evaluation for every bin.
struct Thresholds {
  double th0sq;      // theta0^2
  double rho;
  double eta;
  float t0_lo, t0_hi;              // e0 < t0_lo: T0 fails; e0 > t0_hi: T0 passes (e0 = |s_0|^2 in FP32)
  float t1_hi_pass, t1_hi_fail;    // e <= t1_hi_pass e0: upper T1 bound holds; e > t1_hi_fail e0: fails
  float t1_lo_pass, t1_lo_fail;    // e >= t1_lo_pass e0: lower T1 bound holds; e < t1_lo_fail e0: fails
  float eta_f;
  int fp64_all;
  int amp_average;   // amplitude averaged over the D+1 lines instead of line tau only
};

// Amplitude of a decoded frequency: s_0 W^-p (Eq. decoding), or the mean over the D+1 lines of
// s_j W^-(p + [j > 0] c_{j-1} k_{j-1}) when averaging.  The average is out of line (its operands
// passed by value) so that the option costs the recovery loops no registers when it is off.
template <int D>
struct BinOperands {
  float2 sd[D];
  int k[D];
};

template <int D>
__device__ __noinline__ float2 averaged_amplitude(float2 a0, BinOperands<D> v, const Shape& sh, int p,
                                                  const float2* __restrict__ tw) {
  float2 a = a0;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    int q = p + sh.c[d] * v.k[d];
    if (q >= sh.L) q -= sh.L;
    a = cadd(a, cmul(v.sd[d], tw[q]));
  }
  return cscale(a, 1.0f / (float)(D + 1));
}

template <int D>
__device__ __forceinline__ float2 decoded_amplitude(float2 s0, const float2* sd, const Shape& sh, const int* k, int p,
                                                    const float2* __restrict__ tw, bool average) {
  const float2 a = cmul(s0, tw[p]);
  if (!average) return a;
  BinOperands<D> v;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    v.sd[d] = sd[d];
    v.k[d] = k[d];
  }
  return averaged_amplitude<D>(a, v, sh, p, tw);
}

// Verdicts: 1 = every test passes (k filled), -1 = rejected, 0 = not certified in FP32.
constexpr int kAccept = 1, kReject = -1, kUndecided = 0;

template <int D>
__device__ __forceinline__ int classify_fp32(const float2 s0, const float2* sd, const Shape& sh,
                                             const Thresholds& th, int* k, bool* t0_counted) {
  const float kInvTwoPi = 0.159154943091895336f;
  const float e0 = fmaf(s0.x, s0.x, s0.y * s0.y);
  if (e0 < th.t0_lo) return kReject;               // T0 fails
  if (!(e0 > th.t0_hi)) return kUndecided;
  *t0_counted = true;                              // T0 passes
  bool undecided = false;
#pragma unroll
  for (int d = 0; d < D; ++d) {                    // T1
    const float e = fmaf(sd[d].x, sd[d].x, sd[d].y * sd[d].y);
    if (e > th.t1_hi_fail * e0 || e < th.t1_lo_fail * e0) return kReject;
    if (!(e <= th.t1_hi_pass * e0 && e >= th.t1_lo_pass * e0)) undecided = true;
  }
  if (undecided) return kUndecided;
#pragma unroll
  for (int d = 0; d < D; ++d) {                    // decode + T2
    const float re = fmaf(sd[d].x, s0.x, sd[d].y * s0.y);
    const float im = fmaf(sd[d].y, s0.x, -(sd[d].x * s0.y));
    // FP32 and FP64 may put phi on opposite sides of +-pi; u then differs by N_d, which moves
    // floor(u + 1/2) by N_d and leaves both k_d mod N_d and the distance to the grid unchanged,
    // so the certification below holds modulo N_d.
    const float phi = atan2f(im, re);
    const float nd = (float)sh.dims[d];
    const float u = nd * phi * kInvTwoPi;
    const float r = floorf(u + 0.5f);
    const float dist = fabsf(u - r);
    const float band = 2e-6f * nd + 1e-6f;
    if (fabsf(dist - th.eta_f) <= band || fabsf(dist - 0.5f) <= band) return kUndecided;
    if (dist > th.eta_f) return kReject;
    int kd = (int)r;                               // r in [-N_d/2, N_d/2 + 1]
    if (kd < 0) kd += sh.dims[d];
    if (kd >= sh.dims[d]) kd -= sh.dims[d];
    k[d] = kd;
  }
  return kAccept;
}

// Out of line: it runs only for the rare bins inside a guard band, and keeping its FP64 values
// out of the callers' register allocation lets more CTAs stay resident.
template <int D>
__device__ __noinline__ int classify_fp64(const float2 s0, const float2* sd, const Shape& sh,
                                          const Thresholds& th, int* k, bool* t0_counted) {
  const double kTwoPi = 6.283185307179586476925286766559;
  const double e0 = (double)s0.x * s0.x + (double)s0.y * s0.y;
  if (!(e0 > th.th0sq)) return kReject;                               // T0
  *t0_counted = true;
  const double r0 = sqrt(e0);
  bool ok = true;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    const double e = (double)sd[d].x * sd[d].x + (double)sd[d].y * sd[d].y;
    if (fabs(sqrt(e) - r0) > th.rho * r0) ok = false;                 // T1
  }
  if (!ok) return kReject;
#pragma unroll
  for (int d = 0; d < D; ++d) {
    // phase of s_{d+1} / s_0, taken as the phase of s_{d+1} conj(s_0) (FP64 products are exact)
    const double re = (double)sd[d].x * s0.x + (double)sd[d].y * s0.y;
    const double im = (double)sd[d].y * s0.x - (double)sd[d].x * s0.y;
    const double u = (double)sh.dims[d] * atan2(im, re) / kTwoPi;
    const double r = floor(u + 0.5);
    if (fabs(u - r) > th.eta) ok = false;                             // T2
    int kd = (int)r;                                                  // r in [-N_d/2, N_d/2 + 1]
    if (kd < 0) kd += sh.dims[d];
    if (kd >= sh.dims[d]) kd -= sh.dims[d];
    k[d] = kd;
  }
  return ok ? kAccept : kReject;
}

// Tests T0..T3 on every bin m of the (already peeled) lines; bins of line j at bins[j*line_stride].
// Adds the number of line-0 bins passing T0 to *t0 and of bins decoded (T0..T3 passed) to
// *accepted, and sets *ovf on a capacity overflow.
template <int D>
__device__ __forceinline__ void decode_bins(const float2* bins, int line_stride, const Shape& sh,
                                            const SetView& s, const int* ca, const int* ct,
                                            const float2* __restrict__ tw, const Thresholds& th,
                                            int* t0, int* ovf, int* accepted) {
  const int L = sh.L;
  int my_t0 = 0, my_acc = 0;
  bool my_ovf = false;
  for (int m = threadIdx.x; m < L; m += blockDim.x) {
    const float2 s0 = bins[m];
    float2 sd[D];
#pragma unroll
    for (int d = 0; d < D; ++d) sd[d] = bins[(d + 1) * line_stride + m];
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
    int msum = 0, psum = 0, key = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) {
      msum += ca[d] * k[d];
      psum += ct[d] * k[d];
      key += k[d] * sh.strides[d];
    }
    if (fmod_(msum, sh.fL) != m) continue;                            // T3
    const float2 a = decoded_amplitude<D>(s0, sd, sh, k, fmod_(psum, sh.fL), tw, th.amp_average != 0);
    ++my_acc;
    if (!set_insert<D>(s, k, key, a)) my_ovf = true;
  }
  if (my_t0) atomicAdd(t0, my_t0);
  if (my_acc) atomicAdd(accepted, my_acc);
  if (my_ovf) atomicOr(ovf, 1);
}

// |a|^2 > theta0^2, certified in FP32 when outside the guard band, else in FP64.
__device__ __forceinline__ bool keep_amplitude(float2 a, const Thresholds& th) {
  if (!th.fp64_all) {
    const float e = fmaf(a.x, a.x, a.y * a.y);
    if (e < th.t0_lo) return false;
    if (e > th.t0_hi) return true;
  }
  return (double)a.x * a.x + (double)a.y * a.y > th.th0sq;
}

// ------------------------------------------------------------------------------------------------
// Output: drop |a| <= theta0 and sort by linear index (bitonic sort)
// ------------------------------------------------------------------------------------------------
// Sort (skey, sidx) pairs by key, n of them, CTA-cooperatively; the arrays need pow2ceil(n)
// entries (padding gets the largest key).  Keys are unique, so the order is deterministic.
__device__ __forceinline__ void bitonic_sort_pairs(int* skey, int* sidx, int n) {
  int P = 1;
  while (P < n) P <<= 1;
  for (int i = n + threadIdx.x; i < P; i += blockDim.x) {
    skey[i] = 0x7fffffff;
    sidx[i] = -1;
  }
  __syncthreads();
  for (int k = 2; k <= P; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += blockDim.x) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const bool up = (i & k) == 0;
          const int ki = skey[i], kj = skey[ixj];
          if ((ki > kj) == up) {
            skey[i] = kj;
            skey[ixj] = ki;
            const int t = sidx[i];
            sidx[i] = sidx[ixj];
            sidx[ixj] = t;
          }
        }
      }
      __syncthreads();
    }
  }
}

// Rank sort for n <= 4 blockDim unique keys: the final position of a key is the number of smaller
// keys.  Thread t owns positions t + q blockDim (q < E) and counts over the whole key array with
// broadcast shared-memory reads (16 bytes at a time when skey is 16-byte aligned), so the count
// needs no barrier; the permuted pairs are written back after one.
template <int E>
__device__ __forceinline__ void rank_sort_pairs(int* skey, int* sidx, int n) {
  int mk[E], mi[E], rk[E];
#pragma unroll
  for (int q = 0; q < E; ++q) {
    const int p = threadIdx.x + q * blockDim.x;
    mk[q] = p < n ? skey[p] : 0x7fffffff;
    mi[q] = p < n ? sidx[p] : -1;
    rk[q] = 0;
  }
  if ((int)threadIdx.x < n) {
    int j = 0;
    const bool vec = (reinterpret_cast<uintptr_t>(skey) & 15) == 0;
    for (; vec && j + 4 <= n; j += 4) {
      const int4 v = *reinterpret_cast<const int4*>(skey + j);
#pragma unroll
      for (int q = 0; q < E; ++q)
        rk[q] += (v.x < mk[q] ? 1 : 0) + (v.y < mk[q] ? 1 : 0) + (v.z < mk[q] ? 1 : 0) + (v.w < mk[q] ? 1 : 0);
    }
    for (; j < n; ++j) {
      const int v = skey[j];
#pragma unroll
      for (int q = 0; q < E; ++q) rk[q] += v < mk[q] ? 1 : 0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < E; ++q) {
    if (threadIdx.x + q * blockDim.x < n) {
      skey[rk[q]] = mk[q];
      sidx[rk[q]] = mi[q];
    }
  }
  __syncthreads();
}

// Sort n (skey, sidx) pairs with unique keys by key; the caller has synchronised after writing
// them.  Up to 4 blockDim pairs by rank, more by the bitonic network (pow2ceil(n) entries).
__device__ __forceinline__ void sort_pairs(int* skey, int* sidx, int n) {
  const int E = (n + (int)blockDim.x - 1) / (int)blockDim.x;
  switch (E) {
    case 0: return;
    case 1: rank_sort_pairs<1>(skey, sidx, n); return;
    case 2: rank_sort_pairs<2>(skey, sidx, n); return;
    case 3: rank_sort_pairs<3>(skey, sidx, n); return;
    case 4: rank_sort_pairs<4>(skey, sidx, n); return;
    default: bitonic_sort_pairs(skey, sidx, n); return;
  }
}

// Output in order of linear index through a bitmap of the N grid points held in `region`
// (needs 4 (ceil(N/32) + blockDim) bytes; false: does nothing).  get(i, key, a) says whether entry
// i < count is kept and gives its key and amplitude; put(r, key, a) writes output row r.  The
// position of a kept key is the number of set bits below it: bits set by atomicOr, popcounts
// summed per thread over a contiguous chunk of words, an exclusive scan of the chunk sums by warp
// 0, popcounts inside the chunk.  *n_out = number of entries written.  All threads must call it.
template <typename Get, typename Put>
__device__ __forceinline__ bool emit_by_bitmap(int count, int N, unsigned char* region, size_t region_bytes,
                                               int* n_out, Get get, Put put) {
  const int bd = blockDim.x;
  const int tid = threadIdx.x;
  const int W = (N + 31) >> 5;
  if (((size_t)W + (size_t)bd) * sizeof(unsigned) > region_bytes) return false;
  unsigned* bm = reinterpret_cast<unsigned*>(region);
  int* part = reinterpret_cast<int*>(region + region_bytes) - bd;   // chunk sums, after the bitmap
  for (int w = tid; w < W; w += bd) bm[w] = 0u;
  __syncthreads();
  for (int i = tid; i < count; i += bd) {
    int key;
    float2 a;
    if (get(i, key, a)) atomicOr(&bm[key >> 5], 1u << (key & 31));
  }
  __syncthreads();
  const int chunk = (W + bd - 1) / bd;
  {
    const int w0 = min(W, tid * chunk);
    const int w1 = min(W, w0 + chunk);
    int c = 0;
    for (int w = w0; w < w1; ++w) c += __popc(bm[w]);
    part[tid] = c;
  }
  __syncthreads();
  if (tid < 32) {   // lane l scans the run [l per, (l + 1) per) of chunk sums
    const int per = (bd + 31) >> 5;
    int sum = 0;
    for (int q = 0; q < per; ++q) {
      const int j = tid * per + q;
      if (j < bd) sum += part[j];
    }
    int incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    int run = incl - sum;
    for (int q = 0; q < per; ++q) {
      const int j = tid * per + q;
      if (j < bd) {
        const int v = part[j];
        part[j] = run;
        run += v;
      }
    }
    if (tid == 31) *n_out = incl;
  }
  __syncthreads();
  for (int i = tid; i < count; i += bd) {
    int key;
    float2 a;
    if (get(i, key, a)) {
      const int w = key >> 5;
      const int owner = w / chunk;
      int r = part[owner];
      for (int u = owner * chunk; u < w; ++u) r += __popc(bm[u]);
      r += __popc(bm[w] & ((1u << (key & 31)) - 1u));
      put(r, key, a);
    }
  }
  __syncthreads();
  return true;
}

constexpr int kOutBuckets = 64;

// Output of the kept entries (|a| > theta0, a = amp_of(i)) in order of linear index by a bucket
// sort on the key's top bits (keys < N <= 2^nb, bucket = key >> (nb - 6)): a count per bucket, an
// exclusive scan of the 64 counts by one warp, a scatter into bucket order, and the rank of each
// key inside its bucket by counting the bucket's smaller keys; put(r, i) writes output row r from
// entry i.  tkey / tidx need `count` ints each, s_cnt / s_off kOutBuckets ints.  Returns the
// number written.
template <typename AmpOf, typename KeyOf, typename Put>
__device__ __forceinline__ int emit_bucketed(int count, int N, const Thresholds& th, int* tkey, int* tidx, int* s_cnt,
                                             int* s_off, int* s_n, AmpOf amp_of, KeyOf key_of, Put put) {
  const int tid = threadIdx.x;
  const int bd = blockDim.x;
  int nb = 0;
  while ((1 << nb) < N) ++nb;
  const int shift = nb > 6 ? nb - 6 : 0;
  for (int q = tid; q < kOutBuckets; q += bd) s_cnt[q] = 0;
  __syncthreads();
  for (int i = tid; i < count; i += bd)
    if (keep_amplitude(amp_of(i), th)) atomicAdd(&s_cnt[key_of(i) >> shift], 1);
  __syncthreads();
  if (tid < 32) {   // lane l scans buckets 2l and 2l + 1
    const int c0 = s_cnt[2 * tid], c1 = s_cnt[2 * tid + 1];
    int incl = c0 + c1;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (tid >= o) incl += y;
    }
    const int excl = incl - (c0 + c1);
    s_off[2 * tid] = excl;
    s_off[2 * tid + 1] = excl + c0;
    s_cnt[2 * tid] = 0;         // from here on: fill counters
    s_cnt[2 * tid + 1] = 0;
    if (tid == 31) *s_n = incl;
  }
  __syncthreads();
  for (int i = tid; i < count; i += bd) {
    if (keep_amplitude(amp_of(i), th)) {
      const int key = key_of(i);
      const int bk = key >> shift;
      const int pos = s_off[bk] + atomicAdd(&s_cnt[bk], 1);
      tkey[pos] = key;
      tidx[pos] = i;
    }
  }
  __syncthreads();
  const int n = *s_n;
  for (int p = tid; p < n; p += bd) {
    const int key = tkey[p];
    const int bk = key >> shift;
    const int hi = bk + 1 < kOutBuckets ? s_off[bk + 1] : n;
    int r = s_off[bk];
    for (int q = s_off[bk]; q < hi; ++q) r += tkey[q] < key ? 1 : 0;
    put(r, tidx[p]);
  }
  __syncthreads();
  return n;
}

// Compact the entries with |a| > theta0 into (skey, sidx) and sort them by linear index: on return
// *n_out is the number kept and sidx[r] the list position of the r-th smallest key.
__device__ __forceinline__ void sort_kept(const SetView& s, int count, const Thresholds& th, int* skey, int* sidx,
                                          int* n_out) {
  if (threadIdx.x == 0) *n_out = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    if (keep_amplitude(s.la[i], th)) {
      const int pos = atomicAdd(n_out, 1);
      skey[pos] = s.lkey[i];
      sidx[pos] = i;
    }
  }
  __syncthreads();
  sort_pairs(skey, sidx, *n_out);
}

}  // namespace fpssft

namespace fpssft {

// ------------------------------------------------------------------------------------------------
// Register FFT of one line per warp, for L = 32 R (R = 1, 2, 4, 8, 16)
// ------------------------------------------------------------------------------------------------
// Lane l holds v[i] = s(l + 32 i).  With n = l + 32 i and m = k2 + R k1:
//   s_hat(m) L = sum_l W_32^{l k1} W_L^{l k2} sum_i s(l + 32 i) W_R^{i k2}
// so each lane takes the R-point DFT of its registers, multiplies register k2 by W_L^{l k2}, and
// the warp takes a 32-point DFT across lanes for every k2 (radix-2 decimation in frequency with
// __shfl_xor_sync; the result lands in bit-reversed lane order).  Afterwards lane l holds
// v[k2] = L s_hat(k2 + R brev5(l)).  tw[q] = exp(-j 2 pi q / L).
template <int R>
__device__ __forceinline__ void butterfly_tw(float2 (&v)[R], const float2* __restrict__ tw, int L) {
  butterfly<R>(v);
}

template <>
__device__ __forceinline__ void butterfly_tw<1>(float2 (&v)[1], const float2* __restrict__, int) {}

template <>
__device__ __forceinline__ void butterfly_tw<16>(float2 (&v)[16], const float2* __restrict__ tw, int L) {
  // 16 = 4 x 4: DFTs over i2 (stride 4), twiddle W_16^{i1 k2}, DFTs over i1
  const int q16 = L >> 4;     // W_16^q = tw[q L / 16]
  float2 a[4][4];
#pragma unroll
  for (int i1 = 0; i1 < 4; ++i1) {
    float2 t[4] = {v[i1], v[i1 + 4], v[i1 + 8], v[i1 + 12]};
    butterfly<4>(t);
#pragma unroll
    for (int k2 = 0; k2 < 4; ++k2) a[i1][k2] = (i1 * k2 == 0) ? t[k2] : cmul(t[k2], tw[i1 * k2 * q16]);
  }
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 t[4] = {a[0][k2], a[1][k2], a[2][k2], a[3][k2]};
    butterfly<4>(t);
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) v[k2 + 4 * k1] = t[k1];
  }
}

template <int R>
__device__ __forceinline__ void warp_fft(float2 (&v)[R], const float2* __restrict__ tw, int L, int lane) {
  butterfly_tw<R>(v, tw, L);
#pragma unroll
  for (int k2 = 1; k2 < R; ++k2) v[k2] = cmul(v[k2], tw[lane * k2]);
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
    const float2 w = tw[(lane & (h - 1)) * (L / (2 * h))];
#pragma unroll
    for (int k2 = 0; k2 < R; ++k2) {
      const float px = __shfl_xor_sync(0xffffffffu, v[k2].x, h);
      const float py = __shfl_xor_sync(0xffffffffu, v[k2].y, h);
      if (!upper) {
        v[k2] = make_float2(v[k2].x + px, v[k2].y + py);
      } else {
        v[k2] = cmul(make_float2(px - v[k2].x, py - v[k2].y), w);
      }
    }
  }
}

__device__ __forceinline__ int brev5(int x) { return (int)(__brev((unsigned)x) >> 27); }

// Bank swizzle of a bin index inside aligned groups of 16 (a bijection on [L] for 16 | L): the
// bit-reversed stores of warp_fft then spread over all banks.
__device__ __forceinline__ int swz(int m) { return m ^ ((m >> 4) & 15); }

// Gather line j of iteration (al, ta) into registers: v[i] = x(n_j(lane + 32 i)).
template <int D, int R>
__device__ __forceinline__ void gather_line_regs(float2 (&v)[R], const float2* __restrict__ x, const Shape& sh,
                                                 const int* al, const int* ta, int j, int lane) {
  int n[D], stepn[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    n[d] = fmod_(al[d] * lane + ta[d] + (j == d + 1 ? 1 : 0), sh.fdims[d]);
    stepn[d] = fmod_(al[d] * 32, sh.fdims[d]);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int base = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) base += n[d] * sh.strides[d];
    v[i] = __ldg(x + base);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      n[d] += stepn[d];
      if (n[d] >= sh.dims[d]) n[d] -= sh.dims[d];
    }
  }
}

// Request line j's samples into L2 without waiting for them (prefetch.global.L2).  No register
// receives them, so the CTA barriers that follow do not wait for them as they wait for
// outstanding loads; the next iteration's synchronous gather then finds them in L2.
template <int D, int R>
__device__ __forceinline__ void prefetch_line_l2(const float2* __restrict__ x, const Shape& sh, const int* al,
                                                 const int* ta, int j, int lane) {
  int n[D], stepn[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    n[d] = fmod_(al[d] * lane + ta[d] + (j == d + 1 ? 1 : 0), sh.fdims[d]);
    stepn[d] = fmod_(al[d] * 32, sh.fdims[d]);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int base = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) base += n[d] * sh.strides[d];
    asm volatile("prefetch.global.L2 [%0];" ::"l"(x + base));
#pragma unroll
    for (int d = 0; d < D; ++d) {
      n[d] += stepn[d];
      if (n[d] >= sh.dims[d]) n[d] -= sh.dims[d];
    }
  }
}

// Asynchronous copy of line j's samples into shared memory: lane l copies samples l + 32 i into
// stg[l + 32 i].  After cp.async.wait_group the lane reads back exactly what it copied itself, so
// no barrier is needed.
template <int D, int R>
__device__ __forceinline__ void gather_line_async(float2* stg, const float2* __restrict__ x, const Shape& sh,
                                                  const int* al, const int* ta, int j, int lane) {
  int n[D], stepn[D];
#pragma unroll
  for (int d = 0; d < D; ++d) {
    n[d] = fmod_(al[d] * lane + ta[d] + (j == d + 1 ? 1 : 0), sh.fdims[d]);
    stepn[d] = fmod_(al[d] * 32, sh.fdims[d]);
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int base = 0;
#pragma unroll
    for (int d = 0; d < D; ++d) base += n[d] * sh.strides[d];
    cp_async8(stg + lane + 32 * i, x + base);
#pragma unroll
    for (int d = 0; d < D; ++d) {
      n[d] += stepn[d];
      if (n[d] >= sh.dims[d]) n[d] -= sh.dims[d];
    }
  }
  cp_async_commit();
}

// The recovered set of the warp-FFT kernel: dense list (lk, la) and per-iteration buckets built by
// the peel (head[m] -> first entry whose bin is m, nxt[i] -> next entry of the same bin).  A
// frequency decoded from bin m that is already in the set must lie in bucket m (its bin is m by
// T3), so the buckets replace a hash index.
struct BucketSet {
  int* lk;       // [D][k_cap]
  float2* la;    // [k_cap]
  int* head;     // [L_max]
  int* nxt;      // [k_cap]
  int* count;
  int k_cap;
};

template <int D>
__device__ __forceinline__ bool bucket_insert(const BucketSet& s, int m, const int* k, float2 a) {
  for (int h = s.head[m]; h >= 0; h = s.nxt[h]) {
    bool same = true;
#pragma unroll
    for (int d = 0; d < D; ++d) same = same && s.lk[d * s.k_cap + h] == k[d];
    if (same) {
      s.la[h] = cadd(s.la[h], a);
      return true;
    }
  }
  const int idx = atomicAdd(s.count, 1);
  if (idx >= s.k_cap) return false;
#pragma unroll
  for (int d = 0; d < D; ++d) s.lk[d * s.k_cap + idx] = k[d];
  s.la[idx] = a;
  return true;
}

}  // namespace fpssft
