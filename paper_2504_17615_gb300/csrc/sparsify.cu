// sparsify.cu -- edge sparsification to m_hat edges in expectation (Alg. 1,
// Sec. 4.2).
//
// Weighted threshold sampling: w_t is the m_hat-th heaviest undirected edge
// weight, found by a histogram select over the CSR entries (every undirected
// edge appears twice, so the entry rank is 2 m_hat): one capped pass with
// exact bins for weights below 4095 settles the usual case, otherwise an
// exact three-digit MSD radix select over the 31 weight bits.  Edges heavier
// than w_t are kept, lighter ones dropped, and an edge of weight w_t is kept
// iff h32(key(SPARSE, level, 0), min(u,v), max(u,v)) < T with
// T = floor((m_hat - |E>|) 2^32 / |E=|).  Uniform sampling keeps an edge iff
// its hash is below floor(m_hat 2^32 / m).  Both CSR directions of an edge
// see the same hash, so the result stays symmetric.
//
// Two passes over the entries, each warp walking 32 consecutive rows (one
// contiguous range of entries): the first counts the kept entries of every
// row, a prefix sum turns the counts into the new row offsets, and the second
// takes the same keep decisions again and writes the kept entries of the 32
// rows contiguously from the first row's new offset.
#include "gp_internal.cuh"

#include <algorithm>
#include <utility>

namespace gp {

namespace {

constexpr unsigned FULL = 0xFFFFFFFFu;
constexpr int kCapBins = 4096;

__global__ void k_whist(const int32_t *__restrict__ w, int64_t m2, int cap_mode, int prefix_shift,
                        int prefix, int shift, int nbits, unsigned long long *hist) {
  __shared__ unsigned s_h[kCapBins];
  const int nb = cap_mode ? kCapBins : (1 << nbits);
  for (int t = threadIdx.x; t < nb; t += blockDim.x) s_h[t] = 0;
  __syncthreads();
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int x = w[e];
    int bin;
    if (cap_mode) {
      bin = x < kCapBins - 1 ? x : kCapBins - 1;
    } else {
      if ((int)((unsigned)x >> prefix_shift) != prefix) continue;
      bin = (int)(((unsigned)x >> shift) & ((1u << nbits) - 1));
    }
    atomicAdd(&s_h[bin], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nb; t += blockDim.x)
    if (s_h[t]) atomicAdd(&hist[t], (unsigned long long)s_h[t]);
}

struct KeepArgs {
  const int32_t *xadj, *adjncy, *adjwgt;
  int n;
  int mode;  // 0 keep none, 1 threshold, 2 uniform, 3 keep all, 4 exact-count threshold
  int32_t wt;
  uint64_t T;   // modes 1, 2: 32-bit hash threshold; mode 4: the last kept 64-bit hash
  uint64_t key;
  uint32_t blo, bhi;  // mode 4: the last kept edge among those whose hash equals T
  int32_t *cnt;         // count pass: kept entries per row
  const int32_t *nxadj; // write pass: new row offsets
  int32_t *oadj, *ow;
};

constexpr int kKeepUnroll = 4;

__device__ __forceinline__ bool keep_entry(const KeepArgs &a, int row, int v, int x) {
  if (a.mode == 3) return true;
  if (a.mode == 0) return false;
  const uint32_t lo = (uint32_t)(row < v ? row : v), hi = (uint32_t)(row < v ? v : row);
  if (a.mode == 4) {
    if (x != a.wt) return x > a.wt;
    const uint64_t h = h64(a.key, lo, hi);
    return h < a.T || (h == a.T && (lo < a.blo || (lo == a.blo && hi <= a.bhi)));
  }
  const uint64_t h = h32(a.key, lo, hi);
  if (a.mode == 2) return h < a.T;
  return x > a.wt || (x == a.wt && h < a.T);
}

// WRITE = false: kept entries per row; WRITE = true: the kept entries, compacted.
template <bool WRITE>
__global__ void __launch_bounds__(256) k_keep(KeepArgs a) {
  __shared__ int s_cnt[8][32];
  const int lane = (int)lane_id(), wib = threadIdx.x >> 5;
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int64_t u0 = (int64_t)wid * 32; u0 < a.n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const bool valid = u < a.n;
    const int xe = valid ? a.xadj[u + 1] : 0x7FFFFFFF;
    const int e0 = a.xadj[u0];
    const int last = (int)((a.n - u0) < 32 ? (a.n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    if (!WRITE) s_cnt[wib][lane] = 0;
    int out = WRITE ? a.nxadj[u0] : 0;
    __syncwarp();
    for (int f0 = e0; f0 < e1; f0 += 32 * kKeepUnroll) {
      int e[kKeepUnroll], j[kKeepUnroll], v[kKeepUnroll], x[kKeepUnroll];
#pragma unroll
      for (int r = 0; r < kKeepUnroll; r++) {
        e[r] = f0 + r * 32 + lane;
        int q = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int val = __shfl_sync(FULL, xe, q + step - 1);
          if (val <= e[r]) q += step;
        }
        j[r] = q;
      }
#pragma unroll
      for (int r = 0; r < kKeepUnroll; r++) {
        v[r] = e[r] < e1 ? __ldcs(a.adjncy + e[r]) : 0;
        x[r] = e[r] < e1 ? __ldcs(a.adjwgt + e[r]) : 0;
      }
#pragma unroll
      for (int r = 0; r < kKeepUnroll; r++) {
        const bool k = e[r] < e1 && keep_entry(a, (int)(u0 + j[r]), v[r], x[r]);
        if (WRITE) {
          const unsigned m = __ballot_sync(FULL, k);
          if (k) {
            const int pos = out + __popc(m & lanemask_lt());
            a.oadj[pos] = v[r];
            a.ow[pos] = x[r];
          }
          out += __popc(m);
        } else if (k) {
          atomicAdd(&s_cnt[wib][j[r]], 1);
        }
      }
    }
    if (!WRITE) {
      __syncwarp();
      if (valid) a.cnt[u] = s_cnt[wib][lane];
      __syncwarp();
    }
  }
}

// Exact-count mode: histogram of one digit of the 64-bit hash of the edges of
// weight wt (entries with row < neighbour, so every edge once), restricted to
// the hashes whose bits above the digit equal `prefix`; the same 32-row walk
// as k_keep.
struct HashHistArgs {
  const int32_t *xadj, *adjncy, *adjwgt;
  int n;
  int32_t wt;
  uint64_t key;
  int above;        // bits above the digit (0: no prefix)
  uint64_t prefix;
  int shift, nbits;
  unsigned long long *hist;
  uint32_t *pairs;  // collect mode: (lo, hi) of the edges whose hash equals `prefix`
  int *npairs;
  int cap;
};

template <bool COLLECT>
__global__ void __launch_bounds__(256) k_hash_digit(HashHistArgs a) {
  __shared__ unsigned s_h[2048];
  if (!COLLECT) {
    for (int t = threadIdx.x; t < (1 << a.nbits); t += blockDim.x) s_h[t] = 0;
    __syncthreads();
  }
  const int lane = (int)lane_id();
  const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int64_t u0 = (int64_t)wid * 32; u0 < a.n; u0 += (int64_t)nw * 32) {
    const int64_t u = u0 + lane;
    const int xe = u < a.n ? a.xadj[u + 1] : 0x7FFFFFFF;
    const int e0 = a.xadj[u0];
    const int last = (int)((a.n - u0) < 32 ? (a.n - u0) : 32) - 1;
    const int e1 = __shfl_sync(FULL, xe, last);
    for (int f0 = e0; f0 < e1; f0 += 32) {
      const int e = f0 + lane;
      int q = 0;  // owner: lanes whose row ends at or before e
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const int val = __shfl_sync(FULL, xe, q + step - 1);
        if (val <= e) q += step;
      }
      if (e >= e1) continue;
      const int row = (int)(u0 + q), v = __ldcs(a.adjncy + e);
      if (row >= v || __ldcs(a.adjwgt + e) != a.wt) continue;
      const uint64_t h = h64(a.key, (uint32_t)row, (uint32_t)v);
      if (COLLECT) {
        if (h == a.prefix) {
          const int j = atomicAdd(a.npairs, 1);
          if (j < a.cap) { a.pairs[2 * j] = (uint32_t)row; a.pairs[2 * j + 1] = (uint32_t)v; }
        }
      } else {
        if (a.above > 0 && (h >> (64 - a.above)) != a.prefix) continue;
        atomicAdd(&s_h[(unsigned)(h >> a.shift) & ((1u << a.nbits) - 1u)], 1u);
      }
    }
  }
  if (!COLLECT) {
    __syncthreads();
    for (int t = threadIdx.x; t < (1 << a.nbits); t += blockDim.x)
      if (s_h[t]) atomicAdd(&a.hist[t], (unsigned long long)s_h[t]);
  }
}

// The r-th smallest (1-based) 64-bit hash among the edges of weight wt, and the
// edge that closes the kept prefix when several edges share that hash.
void exact_boundary(gp_ctx *ctx, const DevGraph &g, int32_t wt, uint64_t key, int64_t r, uint64_t *t_out,
                    uint32_t *blo, uint32_t *bhi) {
  const int digits[6][2] = {{53, 11}, {42, 11}, {31, 11}, {20, 11}, {10, 10}, {0, 10}};  // (shift, bits)
  DBuf<unsigned long long> hist(ctx, 2048);
  std::vector<unsigned long long> h(2048);
  HashHistArgs a{g.xadj, g.adjncy, g.adjwgt, g.n, wt, key, 0, 0, 0, 0, hist.get(), nullptr, nullptr, 0};
  const int grid = grid_for(g.n, 256, ctx->num_sms * 16);
  uint64_t prefix = 0;
  int64_t below = 0, equal = 0;
  for (int d = 0; d < 6; d++) {
    a.shift = digits[d][0];
    a.nbits = digits[d][1];
    a.prefix = prefix;
    a.above = 64 - (digits[d][0] + digits[d][1]);
    hist.zero();
    k_hash_digit<false><<<grid, 256, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    const int nb = 1 << a.nbits;
    read_back(ctx, hist.get(), sizeof(unsigned long long) * nb, h.data());
    int b = 0;
    for (; b < nb - 1; b++) {
      if (below + (int64_t)h[b] >= r) break;
      below += (int64_t)h[b];
    }
    prefix = (prefix << a.nbits) | (uint64_t)b;
    equal = (int64_t)h[b];
  }
  *t_out = prefix;
  *blo = 0xFFFFFFFFu;
  *bhi = 0xFFFFFFFFu;
  const int64_t need = r - below;  // edges with hash == prefix to keep, 1 <= need <= equal
  if (need < equal) {  // a 64-bit hash collision inside E=: order the tied edges by their endpoints
    GP_REQUIRE(equal <= (1 << 20), GP_ERR_INVALID, "too many equal hashes in the exact sampler");
    DBuf<uint32_t> pairs(ctx, (size_t)(2 * equal));
    DBuf<int> np(ctx, 1);
    np.zero();
    a.prefix = prefix;
    a.pairs = pairs.get();
    a.npairs = np.get();
    a.cap = (int)equal;
    k_hash_digit<true><<<grid, 256, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
    std::vector<uint32_t> hp((size_t)(2 * equal));
    read_back(ctx, pairs.get(), sizeof(uint32_t) * 2 * equal, hp.data());
    std::vector<std::pair<uint32_t, uint32_t>> ps;
    for (int64_t i = 0; i < equal; i++) ps.emplace_back(hp[2 * i], hp[2 * i + 1]);
    std::sort(ps.begin(), ps.end());
    *blo = ps[(size_t)need - 1].first;
    *bhi = ps[(size_t)need - 1].second;
  }
}

// Selects the entry of descending rank R (1-based) among the weights with a
// three-digit MSD radix select; returns the value and the counts above/equal.
int32_t radix_select_desc(gp_ctx *ctx, const int32_t *w, int64_t m2, int64_t R, int64_t *above,
                          int64_t *equal) {
  const int digits[3][2] = {{20, 11}, {10, 10}, {0, 10}};  // (shift, bits)
  DBuf<unsigned long long> hist(ctx, 2048);
  std::vector<unsigned long long> h(2048);
  int prefix = 0, prefix_shift = 31;
  int64_t acc_above = 0;
  for (int d = 0; d < 3; d++) {
    const int shift = digits[d][0], nbits = digits[d][1], nb = 1 << nbits;
    hist.zero();
    k_whist<<<grid_for(m2, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
        w, m2, 0, prefix_shift, prefix, shift, nbits, hist.get());
    GP_LAUNCH_CHECK();
    read_back(ctx, hist.get(), sizeof(unsigned long long) * nb, h.data());
    int b = nb - 1;
    for (; b > 0; b--) {
      if (acc_above + (int64_t)h[b] >= R) break;
      acc_above += (int64_t)h[b];
    }
    prefix = (prefix << nbits) | b;
    prefix_shift = shift;
    if (d == 2) *equal = (int64_t)h[b];
  }
  *above = acc_above;
  return prefix;
}

}  // namespace

void sparsify_graph(gp_ctx *ctx, const DevGraph &g, int64_t m_hat, int32_t level, uint64_t seed,
                    int mode, DevGraph &out, gp_level_stats *st) {
  ProfScope ps(ctx, PROF_SPARSIFY);
  TraceTimer trace(ctx);
  GP_REQUIRE(mode == GP_SPARSIFY_TWEIGHT || mode == GP_SPARSIFY_UNIFORM || mode == GP_SPARSIFY_TWEIGHT_EXACT,
             GP_ERR_INVALID, "unknown sparsifier mode");
  const int n = g.n;
  const int64_t m2 = g.m2, m = m2 / 2;
  int kmode;
  int32_t wt = 0;
  int64_t ng = 0, ne = 0;
  uint64_t T = 0;
  if (m_hat >= m) kmode = 3;
  else if (m_hat <= 0) kmode = 0;
  else if (mode == GP_SPARSIFY_UNIFORM) {
    kmode = 2;
    T = (uint64_t)(((unsigned __int128)m_hat << 32) / (uint64_t)m);
  } else {
    kmode = 1;
    DBuf<unsigned long long> hist(ctx, kCapBins);
    hist.zero();
    k_whist<<<grid_for(m2, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(g.adjwgt, m2, 1, 31, 0, 0,
                                                                           0, hist.get());
    GP_LAUNCH_CHECK();
    std::vector<unsigned long long> h(kCapBins);
    read_back(ctx, hist.get(), sizeof(unsigned long long) * kCapBins, h.data());
    const int64_t R = 2 * m_hat;  // entry rank of the m_hat-th heaviest undirected edge
    if ((int64_t)h[kCapBins - 1] >= R) {
      int64_t above2 = 0, equal2 = 0;
      wt = radix_select_desc(ctx, g.adjwgt, m2, R, &above2, &equal2);
      ng = above2 / 2;
      ne = equal2 / 2;
    } else {
      int64_t cum = (int64_t)h[kCapBins - 1];
      int b = kCapBins - 2;
      for (; b > 1; b--) {
        if (cum + (int64_t)h[b] >= R) break;
        cum += (int64_t)h[b];
      }
      wt = b;
      ng = cum / 2;
      ne = (int64_t)h[b] / 2;
    }
    T = (uint64_t)(((unsigned __int128)(m_hat - ng) << 32) / (uint64_t)ne);
  }
  const uint64_t key = stream_key(seed, mode == GP_SPARSIFY_UNIFORM ? TAG_UNIFORM : TAG_SPARSE,
                                  (uint32_t)level, 0);
  uint32_t blo = 0, bhi = 0;
  if (kmode == 1 && mode == GP_SPARSIFY_TWEIGHT_EXACT) {
    kmode = 4;
    exact_boundary(ctx, g, wt, key, m_hat - ng, &T, &blo, &bhi);
  }
  KeepArgs a{g.xadj, g.adjncy, g.adjwgt, n, kmode, wt, T, key, blo, bhi, nullptr, nullptr, nullptr, nullptr};
  DBuf<int32_t> cnt(ctx, (size_t)n + 1), total(ctx, 1);
  const int kgrid = grid_for(n, 256, ctx->num_sms * 16);
  GP_CUDA(cudaMemsetAsync(cnt.get() + n, 0, sizeof(int32_t), ctx->stream));
  if (n > 0) {
    a.cnt = cnt.get();
    k_keep<false><<<kgrid, 256, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  out.n = n;
  out.bx.reset(ctx, (size_t)n + 1);
  out.xadj = out.bx.get();
  scan_exclusive_i32(ctx, cnt.get(), out.xadj, n + 1, total.get());
  const int32_t m2_out = read_scalar(ctx, total.get());
  out.m2 = m2_out;
  out.ba.reset(ctx, (size_t)m2_out);
  out.bw.reset(ctx, (size_t)m2_out);
  out.adjncy = out.ba.get();
  out.adjwgt = out.bw.get();
  out.bv.reset(ctx, (size_t)n);
  out.vwgt = out.bv.get();
  if (n > 0 && m2_out > 0) {
    a.nxadj = out.xadj; a.oadj = out.adjncy; a.ow = out.adjwgt;
    k_keep<true><<<kgrid, 256, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  if (n > 0)
    GP_CUDA(cudaMemcpyAsync(out.vwgt, g.vwgt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
  // weights once for the selection (T-Weight only), ids and weights once for the keep test,
  // the kept entries written, row offsets read and written, node weights copied
  prof_bytes(ctx, PROF_SPARSIFY, (kmode == 1 || kmode == 4 ? 4.0 * m2 : 0.0) + 8.0 * m2 + 8.0 * m2_out + 8.0 * (n + 1) + 8.0 * n);
  if (trace.on())
    fprintf(stderr, "[gp sparsify] m2=%lld -> %d ms=%.2f\n", (long long)m2, m2_out, trace.ms());
  if (st) {
    st->omega_t = wt;
    st->n_greater = ng;
    st->n_equal = ne;
    st->threshold = T;
    st->m_next = m2_out / 2;
  }
}

}  // namespace gp
