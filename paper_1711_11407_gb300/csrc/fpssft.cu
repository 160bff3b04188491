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

}  // namespace

// ================================================================================================
// Kernels
// ================================================================================================

#include "recover_common.cuh"
#include "recover_shared.cuh"
#include "recover_warp.cuh"
#include "recover_cluster.cuh"
#include "aux_kernels.cuh"
#include "refine.cuh"

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
  int smem_optin = 227 * 1024;   // opt-in shared memory per CTA of the plan's device
  bool tw_smem = true;
  bool prefetch = true;
  bool warp_path = false;   // k_recover_w (register FFT per line) instead of k_recover
  int warp_mode = 0;        // k_recover_w's request of the next iteration's samples (kWPrefetch, ...)
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

// Mixed-radix stage sequence of an L-point FFT under a radix plan (fpssft_params.radix_plan):
// every plan multiplies out to L; only the order and the split of the power of two differ.
std::vector<int> factorize(int L, int plan) {
  int n = L, e = 0;
  while (n % 2 == 0) { n /= 2; ++e; }
  std::vector<int> two, odd;
  if (plan == 1) {
    for (; e >= 2; e -= 2) two.push_back(4);
    if (e == 1) two.push_back(2);
  } else if (plan == 3) {
    const int fours = e == 1 ? 0 : (e % 3 == 1 ? 2 : (e % 3 == 2 ? 1 : 0));
    for (int q = 0; q < (e - 2 * fours) / 3; ++q) two.push_back(8);
    for (int q = 0; q < fours; ++q) two.push_back(4);
    if (e == 1) two.push_back(2);
  } else {
    for (; e >= 3; e -= 3) two.push_back(8);
    if (e == 2) two.push_back(4);
    if (e == 1) two.push_back(2);
  }
  while (n % 3 == 0) { odd.push_back(3); n /= 3; }
  while (n % 5 == 0) { odd.push_back(5); n /= 5; }
  for (int f = 7; (long long)f * f <= n; f += 2) {
    while (n % f == 0) { odd.push_back(f); n /= f; }
  }
  if (n > 1) odd.push_back(n);
  std::vector<int> r;
  if (plan == 2) {
    r = odd;
    r.insert(r.end(), two.begin(), two.end());
  } else {
    r = two;
    r.insert(r.end(), odd.begin(), odd.end());
  }
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
  if (pr.gather_mode < 0 || pr.gather_mode > 5) return fail(FPSSFT_ERR_INVALID, "gather_mode must be in [0, 5]");
  if (pr.cluster_set < 0 || pr.cluster_set > 2) return fail(FPSSFT_ERR_INVALID, "cluster_set must be in [0, 2]");
  if (pr.fft_path < 0 || pr.fft_path > 3) return fail(FPSSFT_ERR_INVALID, "fft_path must be in [0, 3]");
  if (pr.radix_plan < 0 || pr.radix_plan > 3) return fail(FPSSFT_ERR_INVALID, "radix_plan must be in [0, 3]");
  if (pr.host_cubes < 0 || pr.host_cubes > 1) return fail(FPSSFT_ERR_INVALID, "host_cubes must be 0 or 1");
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
      auto rad = factorize((int)L, pr.radix_plan);
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
  P->smem_optin = optin;
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
      P->warp_mode = pr.gather_mode == 3 ? kWStaged : pr.gather_mode == 4 ? kWNone
                   : pr.gather_mode == 5 ? kWL2Hint : kWPrefetch;
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
    // cluster_set 2: the set in global workspace even when it fits shared memory (smaller CTAs can
    // then share an SM: the autotuner's candidate for batches with more clusters than SMs)
    bool gs = pr.cluster_set == 2;
    CLayout cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, pf_c, gs);
    P->prefetch = pf_c;
    if (cl.total > cap && pf_c) {
      cl = recover_layout_c(D, P->L_max, pr.k_cap, 1 << hb, false, gs);
      P->prefetch = false;
    }
    if (cl.total > cap && !gs) {
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
  if ((e = cudaMemset(P->d_counter, 0, sizeof(int))) != cudaSuccess) return cleanup_fail("clear counter", e);
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
    auto warp_kfn = [&](int wm) -> const void* {
      return wm == kWStaged ? (const void*)k_recover_w<DD, kWStaged>
           : wm == kWNone ? (const void*)k_recover_w<DD, kWNone>
           : wm == kWL2Hint ? (const void*)k_recover_w<DD, kWL2Hint> : (const void*)k_recover_w<DD, kWPrefetch>;
    };
    const void* kfn = P->warp_path ? warp_kfn(P->warp_mode)
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
    // register path, library choice: a batch that the staged-prefetch kernel holds resident at once
    // (latency-bound: a few signals per SM) has each iteration's successor copied into shared memory
    // by cp.async while the current one computes; a larger batch gets no prefetch (throughput: the
    // other CTAs hide the gather's latency)
    if (P->warp_path && P->p.gather_mode == 0) {
      const size_t smem_st = recover_layout_w(DD, P->L_max, P->p.k_cap, true).total;
      int per_sm_st = 0;
      if (smem_st + static_reserve <= (size_t)optin) {
        e2 = ensure_dynamic_smem(warp_kfn(kWStaged), smem_st);
        if (e2 == cudaSuccess)
          e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_st, warp_kfn(kWStaged), P->threads, smem_st);
        if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("staged recovery kernel: ") + cudaGetErrorString(e2));
        if (P->p.ctas_per_sm > 0) per_sm_st = std::min(per_sm_st, P->p.ctas_per_sm);
      }
      if (per_sm_st >= 1 && (long long)batch <= (long long)per_sm_st * P->sm_count) {
        P->warp_mode = kWStaged;
        P->smem = smem_st;
        P->prefetch = true;
        P->grid = std::max(1, batch);
      } else {
        P->warp_mode = kWNone;
        e2 = ensure_dynamic_smem(warp_kfn(P->warp_mode), P->smem);
        if (e2 != cudaSuccess) return fail(FPSSFT_ERR_CUDA, std::string("cudaFuncSetAttribute(recovery kernel): ") + cudaGetErrorString(e2));
      }
    }
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
  RecoverArgs A{};
  A.cubes = static_cast<const float2*>(cubes);
  A.offsets = offsets;
  A.alpha = alpha;
  A.tau = tau;
  A.sched_stride = P->T_max * P->D;
  A.tab = P->tables();
  A.work_counter = P->d_counter;        // zero at plan creation, returned to 0 by every launch
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
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    if (P->warp_path) {
      if (P->warp_mode == kWStaged)
        k_recover_w<DD, kWStaged><<<P->grid, P->threads, P->smem, s>>>(A);
      else if (P->warp_mode == kWNone)
        k_recover_w<DD, kWNone><<<P->grid, P->threads, P->smem, s>>>(A);
      else if (P->warp_mode == kWL2Hint)
        k_recover_w<DD, kWL2Hint><<<P->grid, P->threads, P->smem, s>>>(A);
      else
        k_recover_w<DD, kWPrefetch><<<P->grid, P->threads, P->smem, s>>>(A);
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
  // cubes in pinned host memory the device can address are read in place when the plan asks for it
  const void* in_place = nullptr;
  if (P->p.host_cubes == 1) {
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, cubes) == cudaSuccess && at.type == cudaMemoryTypeHost &&
        at.devicePointer != nullptr)
      in_place = at.devicePointer;
    cudaGetLastError();   // a pointer the runtime does not know is pageable memory: copy it
  }
  if (!in_place && P->st_cubes != nullptr && elems > P->st_cubes_elems) {
    cudaFree(P->st_cubes);
    P->st_cubes = nullptr;
    P->st_cubes_elems = 0;
  }
  if (!in_place && P->st_cubes == nullptr) {
    const size_t n = std::max(elems, P->total_elems);
    if (alloc(&P->st_cubes, n * sizeof(float2)) != cudaSuccess) return fail(FPSSFT_ERR_ALLOC, "staging allocation failed");
    P->st_cubes_elems = n;
  }
  if (P->st_offsets == nullptr) {
    cudaError_t e = cudaSuccess;
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
  if (!in_place)
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
  fpssft_status st = fpssft_recover(P, in_place ? in_place : P->st_cubes, P->st_offsets, P->st_alpha, P->st_tau, dinit,
                                    P->st_k, P->st_a, P->st_count, P->st_iters, P->st_status, stream);
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
                                       int32_t* k, void* a, int32_t* count, int32_t* t0_count, int32_t* accepted,
                                       int32_t* status, void* stream) {
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
  A.accepted = accepted;
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

// ---- least-squares amplitude refinement ---------------------------------------------------------
namespace {
struct RefineLayout {
  size_t r, p, g, sc, total;
};
RefineLayout refine_layout(int batch, int k_cap) {
  auto al = [](size_t v) -> size_t { return (v + 255) & ~size_t(255); };
  RefineLayout w{};
  const size_t vec = (size_t)batch * k_cap * sizeof(float2);
  w.r = 0;
  w.p = al(w.r + vec);
  w.g = al(w.p + vec);
  w.sc = al(w.g + vec);
  w.total = al(w.sc + (size_t)batch * sizeof(RefineScalars));
  return w;
}
}  // namespace

extern "C" fpssft_status fpssft_refine_workspace_size(fpssft_plan_t P, size_t* bytes) {
  if (!P || !bytes) return fail(FPSSFT_ERR_INVALID, "null plan or output");
  *bytes = refine_layout(P->batch, P->p.k_cap).total;
  return FPSSFT_OK;
}

extern "C" fpssft_status fpssft_refine(fpssft_plan_t P, const void* bins, const int32_t* alpha, const int32_t* tau,
                                       int n_sched, const int32_t* k, const int32_t* count, void* a, int iters,
                                       float tol, void* workspace, size_t workspace_bytes, float* resid,
                                       void* stream) {
  if (!P) return fail(FPSSFT_ERR_INVALID, "null plan");
  if (n_sched < 0 || iters < 0) return fail(FPSSFT_ERR_INVALID, "n_sched and iters must be >= 0");
  if (!(tol >= 0.f)) return fail(FPSSFT_ERR_INVALID, "tol must be >= 0");
  if (P->batch == 0) return FPSSFT_OK;
  if (!bins || !alpha || !tau || !k || !count || !a || !workspace) return fail(FPSSFT_ERR_INVALID, "null device pointer");
  const RefineLayout w = refine_layout(P->batch, P->p.k_cap);
  if (workspace_bytes < w.total) return fail(FPSSFT_ERR_INVALID, "workspace smaller than fpssft_refine_workspace_size");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255) != 0) return fail(FPSSFT_ERR_INVALID, "workspace must be 256-byte aligned");
  const size_t lines = (size_t)(P->D + 1) * P->L_max * sizeof(float2);
  const size_t with_g = lines + (size_t)P->p.k_cap * sizeof(float2);
  const size_t reserve = sizeof(Shape) + 512;
  if (lines + reserve > (size_t)P->smem_optin) return fail(FPSSFT_ERR_UNSUPPORTED, "lines of this plan exceed one CTA's shared memory");
  const bool g_in_smem = with_g + reserve <= (size_t)P->smem_optin;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned char* ws = static_cast<unsigned char*>(workspace);
  float2* r = reinterpret_cast<float2*>(ws + w.r);
  float2* pv = reinterpret_cast<float2*>(ws + w.p);
  float2* g = reinterpret_cast<float2*>(ws + w.g);
  RefineScalars* sc = reinterpret_cast<RefineScalars*>(ws + w.sc);
  FPSSFT_CUDA_TRY(cudaMemsetAsync(ws + w.g, 0, w.total - w.g, s));

  RefineNormalArgs N{};
  N.y = static_cast<const float2*>(bins);
  N.alpha = alpha;
  N.tau = tau;
  N.n_sched = n_sched;
  N.tab = P->tables();
  N.batch = P->batch;
  N.L_max = P->L_max;
  N.k_cap = P->p.k_cap;
  N.k = k;
  N.count = count;
  N.g = g;
  N.sc = sc;
  N.g_in_smem = g_in_smem ? 1 : 0;
  // rows split so that about four CTAs per SM have work
  const long long want = (long long)P->sm_count * 4;
  const int ups = (int)std::max(1LL, std::min<long long>(n_sched, (want + P->batch - 1) / P->batch));
  N.units_per_signal = ups;
  N.rows_per_unit = n_sched > 0 ? (n_sched + ups - 1) / ups : 1;
  const int ngrid = unit_grid(P, (long long)P->batch * ups, 8);
  const size_t nsm = g_in_smem ? with_g : lines;
  RefineUpdateArgs U{};
  U.batch = P->batch;
  U.k_cap = P->p.k_cap;
  U.count = count;
  U.a = static_cast<float2*>(a);
  U.r = r;
  U.p = pv;
  U.g = g;
  U.sc = sc;
  U.resid = resid;
  U.tol2 = (double)tol * (double)tol;
  const int ugrid = unit_grid(P, P->batch, 8);
  return dispatch_D(P->D, [&](auto Dc) -> fpssft_status {
    constexpr int DD = decltype(Dc)::value;
    FPSSFT_CUDA_TRY(ensure_dynamic_smem((const void*)k_refine_normal<DD>, nsm));
    auto normal = [&](int mode, const float2* v, int want_g) -> cudaError_t {
      N.mode = mode;
      N.v = v;
      N.want_g = want_g;
      k_refine_normal<DD><<<ngrid, 256, nsm, s>>>(N);
      return cudaGetLastError();
    };
    auto update = [&](int mode) -> cudaError_t {
      U.mode = mode;
      k_refine_update<<<ugrid, 256, 0, s>>>(U);
      return cudaGetLastError();
    };
    FPSSFT_CUDA_TRY(normal(0, U.a, 1));          // g = S^H (y - S a0)
    FPSSFT_CUDA_TRY(update(0));                  // r = p = g
    for (int it = 0; it < iters; ++it) {
      FPSSFT_CUDA_TRY(normal(1, pv, 1));         // g = S^H S p, sq = ||S p||^2
      FPSSFT_CUDA_TRY(update(1));
    }
    FPSSFT_CUDA_TRY(normal(0, U.a, 0));          // sq = ||y - S a||^2
    FPSSFT_CUDA_TRY(update(2));
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

extern "C" fpssft_status fpssft_fft_stages(int L, int radix_plan, int32_t* radices, int32_t* n_stages) {
  if (!radices || !n_stages) return fail(FPSSFT_ERR_INVALID, "null output");
  if (L < 1 || L > (1 << 24)) return fail(FPSSFT_ERR_INVALID, "L must be in [1, 2^24]");
  if (radix_plan < 0 || radix_plan > 3) return fail(FPSSFT_ERR_INVALID, "radix_plan must be in [0, 3]");
  const std::vector<int> r = factorize(L, radix_plan);
  if ((int)r.size() > kMaxStages) return fail(FPSSFT_ERR_UNSUPPORTED, "too many FFT stages");
  for (size_t i = 0; i < r.size(); ++i) radices[i] = r[i];
  *n_stages = (int32_t)r.size();
  return FPSSFT_OK;
}

extern "C" const char* fpssft_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* fpssft_version(void) { return "fpssft-gb300 0.1 (sm_103a)"; }

static_assert(kNumPhases == FPSSFT_PHASE_COUNT && kPhaseWords == FPSSFT_PHASE_WORDS, "phase counter layout");

extern "C" fpssft_status fpssft_phase_read(int64_t* out) {
#ifdef FPSSFT_PHASE_TIMERS
  if (!out) return fail(FPSSFT_ERR_INVALID, "null output");
  unsigned long long h[kPhaseWords];
  const unsigned long long z[kPhaseWords] = {};
  FPSSFT_CUDA_TRY(cudaDeviceSynchronize());
  FPSSFT_CUDA_TRY(cudaMemcpyFromSymbol(h, g_phase, sizeof(h)));
  FPSSFT_CUDA_TRY(cudaMemcpyToSymbol(g_phase, z, sizeof(z)));
  for (int i = 0; i < kPhaseWords; ++i) out[i] = (int64_t)h[i];
  return FPSSFT_OK;
#else
  (void)out;
  return fail(FPSSFT_ERR_UNSUPPORTED, "library built without FPSSFT_PHASE_TIMERS");
#endif
}

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

// The tables reach the array inside kernel parameters: the driver copies a launch's parameters
// when the launch is issued, so the call reads no host memory after it returns and does not wait
// for the stream's earlier work (a copy from pageable host memory would do both).  One launch
// carries up to kUploadBytes (the parameter space holds 32 764 bytes); destinations and sizes
// are multiples of 16 bytes.
constexpr int kUploadBytes = 32000;

struct UploadChunk {
  uint4 data[kUploadBytes / 16];
  uint4* dst;
  int n16;              // 16-byte words to copy
  int* clear;           // an int to set to zero first (nullable)
};

__global__ void __launch_bounds__(256) k_noalloc_upload(const __grid_constant__ UploadChunk c) {
  if (c.clear != nullptr && threadIdx.x == 0) *c.clear = 0;
  for (int i = threadIdx.x; i < c.n16; i += blockDim.x) c.dst[i] = c.data[i];
}

int factorize_into(int L, int plan, int* out) {
  const std::vector<int> r = factorize(L, plan);
  if ((int)r.size() > kMaxStages) return -1;
  for (size_t s = 0; s < r.size(); ++s) out[s] = r[s];
  return (int)r.size();
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
  if (pr.gather_mode < 0 || pr.gather_mode > 5) return fail(FPSSFT_ERR_INVALID, "gather_mode must be in [0, 5]");
  if (pr.threads < 0 || pr.threads > 512 || (pr.threads % 32) != 0) return fail(FPSSFT_ERR_INVALID, "threads must be a multiple of 32 in [0, 512]");
  if (pr.radix_plan < 0 || pr.radix_plan > 3) return fail(FPSSFT_ERR_INVALID, "radix_plan must be in [0, 3]");

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
      const int nst = factorize_into((int)L, pr.radix_plan, sh.radix);
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

  // ---- upload the tables and clear the work counter (no allocation: kernel parameters) ----------
  const size_t bytes = (off_tw + tw_used * sizeof(float2) + 15) & ~size_t(15);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (size_t at = off_shapes; at < bytes; at += kUploadBytes) {
    static UploadChunk chunk;   // static: 32 KB is too much for the caller's stack; under the mutex
    const size_t n = std::min((size_t)kUploadBytes, bytes - at);
    std::memcpy(chunk.data, g_noalloc_host + at, n);
    chunk.dst = reinterpret_cast<uint4*>(dscratch + at);
    chunk.n16 = (int)(n / 16);
    chunk.clear = at == off_shapes ? reinterpret_cast<int*>(dscratch + off_counter) : nullptr;
    k_noalloc_upload<<<1, 256, 0, s>>>(chunk);
    FPSSFT_CUDA_TRY(cudaGetLastError());
  }

  RecoverArgs A{};
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
