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
// Keep decisions are packed into one bit per entry (a 32-entry word per warp
// step), a prefix sum over word counts gives every kept entry its position,
// and the kept entries are compacted in one flat pass.
#include "gp_internal.cuh"

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
  int64_t m2;
  int mode;  // 0 keep none, 1 threshold, 2 uniform, 3 keep all
  int32_t wt;
  uint64_t T;
  uint64_t key;
  uint32_t *words;
  int32_t *wcnt;
};

constexpr int kWordsPerChunk = 32;

__global__ void __launch_bounds__(256) k_keep_bits(KeepArgs a) {
  const int lane = (int)lane_id();
  const int64_t nwords = (a.m2 + 31) / 32;
  const int64_t nchunks = (nwords + kWordsPerChunk - 1) / kWordsPerChunk;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t c = wid; c < nchunks; c += nw) {
    const int64_t w0 = c * kWordsPerChunk;
    const int64_t w1 = w0 + kWordsPerChunk < nwords ? w0 + kWordsPerChunk : nwords;
    int row = 0;
    if (lane == 0) row = row_of(a.xadj, a.n, w0 * 32);
    row = __shfl_sync(FULL, row, 0);
    for (int64_t wi = w0; wi < w1; wi++) {
      const int64_t e = wi * 32 + lane;
      bool keep = false;
      if (e < a.m2) {
        while (row < a.n - 1 && (int64_t)a.xadj[row + 1] <= e) row++;
        if (a.mode == 3) {
          keep = true;
        } else if (a.mode != 0) {
          const int v = a.adjncy[e];
          const uint32_t lo = (uint32_t)(row < v ? row : v), hi = (uint32_t)(row < v ? v : row);
          const uint64_t h = h32(a.key, lo, hi);
          if (a.mode == 2) {
            keep = h < a.T;
          } else {
            const int x = a.adjwgt[e];
            keep = x > a.wt || (x == a.wt && h < a.T);
          }
        }
      }
      const unsigned m = __ballot_sync(FULL, keep);
      if (lane == 0) {
        a.words[wi] = m;
        a.wcnt[wi] = __popc(m);
      }
    }
  }
}

__global__ void k_new_xadj(const int32_t *xadj, int n, int64_t m2, const uint32_t *words,
                           const int32_t *woff, int32_t total, int32_t *out) {
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r <= n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = xadj[r];
    if (e >= m2) { out[r] = total; continue; }
    const int64_t wi = e >> 5;
    const unsigned b = (unsigned)(e & 31);
    out[r] = woff[wi] + __popc(words[wi] & ((1u << b) - 1u));
  }
}

__global__ void __launch_bounds__(256) k_compact(const int32_t *adjncy, const int32_t *adjwgt, int64_t m2,
                                                 const uint32_t *words, const int32_t *woff,
                                                 int32_t *oadj, int32_t *ow) {
  const int lane = (int)lane_id();
  const int64_t nwords = (m2 + 31) / 32;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t wi = wid; wi < nwords; wi += nw) {
    const unsigned m = words[wi];
    if (!((m >> lane) & 1u)) continue;
    const int64_t e = wi * 32 + lane;
    const int pos = woff[wi] + __popc(m & lanemask_lt());
    oadj[pos] = adjncy[e];
    ow[pos] = adjwgt[e];
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
  GP_REQUIRE(mode == GP_SPARSIFY_TWEIGHT || mode == GP_SPARSIFY_UNIFORM, GP_ERR_INVALID,
             "unknown sparsifier mode");
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
  const int64_t nwords = (m2 + 31) / 32;
  DBuf<uint32_t> words(ctx, (size_t)(nwords > 0 ? nwords : 1));
  DBuf<int32_t> wcnt(ctx, (size_t)(nwords > 0 ? nwords : 1)), woff(ctx, (size_t)(nwords > 0 ? nwords : 1));
  DBuf<int32_t> total(ctx, 1);
  if (nwords > 0) {
    KeepArgs a{g.xadj, g.adjncy, g.adjwgt, n, m2, kmode, wt, T, key, words.get(), wcnt.get()};
    const int64_t chunks = (nwords + kWordsPerChunk - 1) / kWordsPerChunk;
    k_keep_bits<<<grid_for(chunks * 32, 256, ctx->num_sms * 16), 256, 0, ctx->stream>>>(a);
    GP_LAUNCH_CHECK();
  }
  scan_exclusive_i32(ctx, wcnt.get(), woff.get(), nwords, total.get());
  const int32_t m2_out = read_scalar(ctx, total.get());
  out.allocate(ctx, n, m2_out);
  k_new_xadj<<<grid_for((int64_t)n + 1, 256, ctx->num_sms * 8), 256, 0, ctx->stream>>>(
      g.xadj, n, m2, words.get(), woff.get(), m2_out, out.xadj);
  GP_LAUNCH_CHECK();
  if (nwords > 0) {
    k_compact<<<grid_for(nwords * 32, 256, ctx->num_sms * 16), 256, 0, ctx->stream>>>(
        g.adjncy, g.adjwgt, m2, words.get(), woff.get(), out.adjncy, out.adjwgt);
    GP_LAUNCH_CHECK();
  }
  if (n > 0)
    GP_CUDA(cudaMemcpyAsync(out.vwgt, g.vwgt, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, ctx->stream));
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
