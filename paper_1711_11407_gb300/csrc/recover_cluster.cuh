// The cluster recovery kernel k_recover_c (one CTA per line, a thread-block cluster per signal).
// Part of the FPS-SFT recovery library for GB300 (sm_103a), arXiv 1711.11407; included by fpssft.cu.
#pragma once

#include <cooperative_groups.h>

#include "recover_common.cuh"

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
  __shared__ int s_cnt[kOutBuckets], s_off[kOutBuckets];
  __shared__ int s_t0[2];                     // line-0 bins passing T0, by iteration parity
  __shared__ int s_acc[2];                    // bins decoded, by iteration parity
  __shared__ int s_ca[kMaxD], s_ct[kMaxD];
  __shared__ unsigned char* s_base[kMaxD + 1];  // each rank's dynamic shared memory (generic address)

  const int rank = (int)cluster.block_rank();
  FPSSFT_PH_START();
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
    s_acc[0] = 0;
    s_acc[1] = 0;
  }
  cluster.sync();   // every CTA started and initialised before any remote access

  int* c_count = GS ? g_count : cluster.map_shared_rank(&s_count, 0);
  int* c_ovf = cluster.map_shared_rank(&s_ovf, 0);
  int* c_t0 = cluster.map_shared_rank(s_t0, 0);
  int* c_acc = cluster.map_shared_rank(s_acc, 0);
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
  FPSSFT_PH(kPhSetup);
  if (pf && T > 0) gather_one_line<D, 0, true>(bufA, x, sh, sched_a, sched_t, rank);
  int iters = 0;
  for (int t = 0; t < T; ++t) {
    const int par = t & 1;
    const int* al = sched_a + t * D;
    const int* ta = sched_t + t * D;
    // slot par was last read after the decode barrier of iteration t-2, before every rank
    // arrived at the peel barrier of t-1, which this rank has passed
    if (rank == 0 && threadIdx.x == 0) {
      s_t0[par] = 0;
      s_acc[par] = 0;
    }
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
    FPSSFT_PH(kPhGather);
    float2* bins = fft_line(cur, bufB, sh, tws, stws, 1.0f / (float)L);
    FPSSFT_PH(kPhFft);
    peel_line_keys<D, GS>(bins, sh, la, lkey, n_set, s_ca, s_ct, tws, rank);
    FPSSFT_PH(kPhPeel);
    cluster.sync();   // every line peeled
    FPSSFT_PH(kPhExchange);

    const size_t boff = reinterpret_cast<unsigned char*>(bins) - smem;
    int my_t0 = 0, my_acc = 0;
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
      ++my_acc;
      const bool ok = GS ? cluster_insert_g<D>(g_la, g_lkey, g_hkey, g_hidx, g_count, A.k_cap, A.hash_bits, key, a)
                         : cluster_insert<D>(s_base, lay, c_count, A.k_cap, A.hash_bits, rank, key, a);
      if (!ok) my_ovf = true;
    }
    if (my_t0) atomicAdd(c_t0 + par, my_t0);
    if (my_acc) atomicAdd(c_acc + par, my_acc);
    if (my_ovf) atomicOr(c_ovf, 1);
    FPSSFT_PH(kPhDecode);
    cluster.sync();   // every insert landed in every replica
    FPSSFT_PH(kPhExchange);
    n_set = min(GS ? __ldcg(g_count) : *c_count, A.k_cap);
    iters = t + 1;
    if ((A.early_stop && c_t0[par] == 0) || *c_ovf != 0 || (A.early_stop == 2 && c_acc[par] == c_t0[par]))
      break;   // the same verdict on every rank
  }
  if (pf) cp_async_wait<0>();
  cluster.sync();   // no rank reads another's shared memory past this point
  FPSSFT_PH(kPhExchange);
  FPSSFT_PH_ITERS(iters);

  if (rank != 0) {
    FPSSFT_PH_FLUSH();
    return;
  }
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
      FPSSFT_PH(kPhOutput);
      FPSSFT_PH_FLUSH();
      return;
    }
  }
  int P = 1;
  while (P < A.k_cap) P <<= 1;
  // otherwise a bucket sort; its buffers: the line buffers, free now, or (GS) the global index
  int* tkey = GS ? g_hkey : reinterpret_cast<int*>(smem + lay.sort);
  int* tidx = GS ? g_hidx : tkey + P;
  auto amp_of = [&](int i) { return GS ? __ldcg(la + i) : la[i]; };
  auto key_of = [&](int i) { return GS ? __ldcg(lkey + i) : lkey[i]; };
  auto put_row = [&](int r, int i) {
    int k[D];
    key_to_k<D>(sh, key_of(i), k);
#pragma unroll
    for (int d = 0; d < D; ++d) ok_out[r * D + d] = k[d];
    oa_out[r] = amp_of(i);
  };
  const int n = emit_bucketed(n_set, sh.N, A.th, tkey, tidx, s_cnt, s_off, &s_n, amp_of, key_of, put_row);
  if (threadIdx.x == 0) {
    A.out_count[b] = n;
    A.out_iters[b] = iters;
    A.out_status[b] = s_ovf ? kStatusCapacity : 0;
  }
  FPSSFT_PH(kPhOutput);
  FPSSFT_PH_FLUSH();
}
