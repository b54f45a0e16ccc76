// love_batch.cu -- batches of independent KISS-GPs (not in the paper: a
// serving form of the LOVE test phase for many GPs of uneven n, m and t).
//
//   love_precompute_batched  B pre-computes at once, one per stream of a
//                            library-owned pool, driven by host worker threads
//                            (each pre-compute synchronises its own stream)
//   love_predict_batched     every GP's test points in ONE persistent launch:
//                            a chunk list (rows of one GP each) walked by a
//                            grid of ctas_per_sm x SMs CTAs; the launch shape
//                            (lanes per point, CTAs per SM) is autotuned at
//                            love_batch_create on synthetic in-domain points
//   love_sample_batched      the single-GP sampler per GP on one stream, with
//                            batch-owned work space (no allocation per call)
//   love_batch_serve         predict + sample, optionally captured into one
//                            CUDA graph and replayed
#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>
#include <thread>
#include <vector>

#include "love_internal.cuh"

using namespace love;

struct love_batch {
  int B = 0, dim = 1;
  love_dtype dtype = LOVE_F32, cache_dtype = LOVE_F32;
  std::vector<love_cache*> caches;
  std::vector<int64_t> t_off;  // B + 1 (host)
  Allocator alloc;
  void* d_desc = nullptr;
  size_t desc_bytes = 0;
  int64_t* d_toff = nullptr;
  PredChunk* d_chunks = nullptr;
  int nchunks = 0;
  int lanes = 8, ctas = 8;
  int n_cand = 0;
  float cand_ms[16] = {};
  // sampling work space, shared by the GPs (they run in stream order)
  int ws_s = -1;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // captured serve graph, the stream it runs on (the caller's stream may be
  // the legacy default stream, which cannot be captured; the graph stream is
  // joined to the caller's by events) and the arguments it was captured with
  cudaGraphExec_t gexec = nullptr;
  int64_t gcaptures = 0;          // graphs captured by love_batch_serve
  int64_t gcaptures_dropped = 0;  // of them, dropped because the work space moved
  cudaStream_t gstream = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  const void* gx = nullptr;
  void *gmean = nullptr, *gvar = nullptr, *gsamples = nullptr;
  int gs = -1;
  uint64_t gseed = 0;
};

namespace {

constexpr int64_t kChunkRows = 1024;   // rows per chunk of the batched predict
constexpr int kMaxWorkers = 32;

size_t elem_of(love_dtype d) { return d == LOVE_F64 ? 8 : 4; }

// library-owned streams for concurrent pre-computes (kept for the process's
// lifetime, so allocators that pool memory per stream see stable streams)
std::mutex g_pool_mu;
std::vector<cudaStream_t> g_pool;

love_status pool_streams(int n, std::vector<cudaStream_t>& out) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  while ((int)g_pool.size() < n) {
    cudaStream_t s = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_check(e);
    g_pool.push_back(s);
  }
  out.assign(g_pool.begin(), g_pool.begin() + n);
  return LOVE_OK;
}

love_status batch_predict(love_batch* b, const void* x, void* mean, void* var, int lanes, int ctas, cudaStream_t s) {
  return predict_batched_launch(b->d_desc, b->d_toff, b->d_chunks, b->nchunks, b->dim, b->dtype, b->cache_dtype,
                                lanes, ctas, x, mean, var, s);
}

love_status batch_sample(love_batch* b, const void* x, int s_count, uint64_t seed, void* out, cudaStream_t s) {
  const size_t el = elem_of(b->dtype);
  for (int i = 0; i < b->B; ++i) {
    const int64_t off = b->t_off[i], t = b->t_off[i + 1] - off;
    if (t == 0) continue;
    LOVE_TRY(sample_launch_ws(b->caches[i], t, (const char*)x + (size_t)off * b->dim * el, s_count, seed + i,
                              (char*)out + (size_t)off * s_count * el, b->ws, s));
  }
  return LOVE_OK;
}

love_status ensure_ws(love_batch* b, int s_count, cudaStream_t s) {
  if (b->ws_s == s_count) return LOVE_OK;
  size_t need = 16;
  for (int i = 0; i < b->B; ++i)
    need = std::max(need, sample_ws_bytes(b->caches[i], b->t_off[i + 1] - b->t_off[i], s_count));
  if (need > b->ws_bytes) {
    // love_batch_serve's graph has the old buffer's address baked into its
    // sample launches: let a replay in flight finish, then drop the graph so
    // the next serve call captures again with the new buffer
    if (b->gexec) {
      if (b->gstream) LOVE_CUDA(cudaStreamSynchronize(b->gstream));
      cudaGraphExecDestroy(b->gexec);
      b->gexec = nullptr;
      ++b->gcaptures_dropped;
    }
    if (b->ws) b->alloc.free(b->ws, b->ws_bytes, s);
    b->ws = b->alloc.alloc(need, s);
    b->ws_bytes = b->ws ? need : 0;
    if (!b->ws) {
      b->ws_s = -1;
      return LOVE_ERR_OOM;
    }
  }
  b->ws_s = s_count;
  return LOVE_OK;
}

// Synthetic test points for the autotuner: uniform in each GP's interpolable
// interior (a splitmix64 stream), in the data dtype.
template <typename R>
void synth_points(const love_batch* b, std::vector<R>& x) {
  x.resize((size_t)b->t_off[b->B] * b->dim);
  uint64_t st = 0x5DEECE66Dull;
  for (int i = 0; i < b->B; ++i) {
    const GridHost& g = b->caches[i]->grid;
    for (int64_t p = b->t_off[i]; p < b->t_off[i + 1]; ++p)
      for (int e = 0; e < b->dim; ++e) {
        st += 0x9E3779B97F4A7C15ull;
        uint64_t z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
        const double lo = g.lo[e] + 1.5 * g.h[e], hi = g.lo[e] + (double)(g.g[e] - 3) * g.h[e];
        x[(size_t)p * b->dim + e] = (R)(lo + u * (hi - lo));
      }
  }
}

// time every (lanes, ctas) candidate on synthetic points; keep the fastest
love_status autotune(love_batch* b, cudaStream_t s) {
  const int64_t T = b->t_off[b->B];
  int cand[4];
  const int nl = predict_lane_candidates(b->dim, cand);
  static const int ctas[3] = {4, 8, 16};
  b->lanes = cand[nl > 1 ? 1 : 0];
  b->ctas = 8;
  b->n_cand = 0;
  if (T == 0 || b->nchunks == 0) return LOVE_OK;
  const size_t el = elem_of(b->dtype);
  void* dx = b->alloc.alloc((size_t)T * b->dim * el, s);
  void* dv = b->alloc.alloc((size_t)T * el, s);
  if (!dx || !dv) {
    b->alloc.free(dx, (size_t)T * b->dim * el, s);
    b->alloc.free(dv, (size_t)T * el, s);
    return LOVE_ERR_OOM;
  }
  love_status rc = LOVE_OK;
  if (b->dtype == LOVE_F64) {
    std::vector<double> hx;
    synth_points(b, hx);
    rc = cuda_check(cudaMemcpyAsync(dx, hx.data(), hx.size() * sizeof(double), cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  } else {
    std::vector<float> hx;
    synth_points(b, hx);
    rc = cuda_check(cudaMemcpyAsync(dx, hx.data(), hx.size() * sizeof(float), cudaMemcpyHostToDevice, s));
    if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == LOVE_OK) rc = cuda_check(cudaEventCreate(&e0));
  if (rc == LOVE_OK) rc = cuda_check(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int li = 0; li < nl && rc == LOVE_OK; ++li)
    for (int ci = 0; ci < 3 && rc == LOVE_OK; ++ci) {
      rc = batch_predict(b, dx, nullptr, dv, cand[li], ctas[ci], s);  // warm-up
      if (rc != LOVE_OK) break;
      cudaEventRecord(e0, s);
      const int reps = 3;
      for (int r = 0; r < reps && rc == LOVE_OK; ++r) rc = batch_predict(b, dx, nullptr, dv, cand[li], ctas[ci], s);
      cudaEventRecord(e1, s);
      if (rc != LOVE_OK) break;
      rc = cuda_check(cudaEventSynchronize(e1));
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      ms /= reps;
      if (b->n_cand < 16) b->cand_ms[b->n_cand++] = ms;
      if (ms < best) {
        best = ms;
        b->lanes = cand[li];
        b->ctas = ctas[ci];
      }
    }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // the synthetic points may have set clamp counters: clear the GPs' device status
  for (int i = 0; i < b->B && rc == LOVE_OK; ++i)
    rc = cuda_check(cudaMemsetAsync(b->caches[i]->status, 0, sizeof(DevStatus), s));
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  b->alloc.free(dx, (size_t)T * b->dim * el, s);
  b->alloc.free(dv, (size_t)T * el, s);
  return rc;
}

void batch_free(love_batch* b, cudaStream_t s) {
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->gstream) {
    cudaStreamSynchronize(b->gstream);
    cudaStreamDestroy(b->gstream);
  }
  if (b->gev_in) cudaEventDestroy(b->gev_in);
  if (b->gev_out) cudaEventDestroy(b->gev_out);
  b->alloc.free(b->d_desc, b->desc_bytes * std::max(b->B, 1), s);
  b->alloc.free(b->d_toff, sizeof(int64_t) * (b->B + 1), s);
  b->alloc.free(b->d_chunks, sizeof(PredChunk) * std::max(b->nchunks, 1), s);
  b->alloc.free(b->ws, b->ws_bytes, s);
  cudaStreamSynchronize(s);
  delete b;
}

}  // namespace

extern "C" {

love_status love_precompute_batched(int B, const love_ski_t* skis, const love_precompute_opts* opts, int workers,
                                    love_stream_t stream, love_cache_t* caches, int* k_eff) try {
  if (B < 0 || (B > 0 && (!skis || !opts || !caches))) return LOVE_ERR_ARG;
  for (int b = 0; b < B; ++b) caches[b] = nullptr;
  for (int b = 0; b < B; ++b)
    if (!skis[b]) return LOVE_ERR_ARG;
  if (B == 0) return LOVE_OK;
  const int nw = std::max(1, std::min({workers <= 0 ? 8 : workers, kMaxWorkers, B}));
  std::vector<cudaStream_t> st;
  LOVE_TRY(pool_streams(nw, st));
  cudaStream_t s0 = (cudaStream_t)stream;
  int dev = 0;
  LOVE_CUDA(cudaGetDevice(&dev));
  cudaEvent_t fork = nullptr;
  LOVE_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  LOVE_CUDA(cudaEventRecord(fork, s0));
  for (int w = 0; w < nw; ++w) LOVE_CUDA(cudaStreamWaitEvent(st[w], fork, 0));
  std::vector<love_status> rc(B, LOVE_OK);
  std::vector<int> ke(B, 0);
  // 1-D FP32 batches: the B Lanczos runs as one batched run on the first pool
  // stream (capturable), then the remaining phases per GP on the workers
  bool batched = !(opts->flags & LOVE_BATCH_STREAMS);
  for (int b = 0; b < B && batched; ++b) {
    const love_ski* k = skis[b];
    batched = k->dtype == LOVE_F32 && k->grid.dim == 1 && !k->grid.additive &&
              precompute_opts_check(k, opts) == LOVE_OK;
  }
  std::vector<float*> Qb(B, nullptr);
  std::vector<int> kb(B, 0);
  BatchedLanczos bl;
  auto free_q = [&]() {
    for (int b = 0; b < B; ++b)
      if (Qb[b]) skis[b]->alloc.free(Qb[b], sizeof(float) * (size_t)skis[b]->n_pad * kb[b], st[0]);
    for (int b = 0; b < B; ++b) Qb[b] = nullptr;
  };
  if (batched) {
    double tau = 0.0, eta = 0.0;
    precompute_lanczos_params(skis[0], opts, &tau, &eta);
    love_status brc = LOVE_OK;
    for (int b = 0; b < B && brc == LOVE_OK; ++b) {
      kb[b] = precompute_k(skis[b], opts);
      Qb[b] = (float*)skis[b]->alloc.alloc(sizeof(float) * (size_t)skis[b]->n_pad * kb[b], st[0]);
      if (!Qb[b]) brc = LOVE_ERR_OOM;
    }
    if (brc == LOVE_OK) brc = lanczos_batched(B, skis, kb.data(), Qb.data(), tau, eta, 0, st[0], &bl);
    if (brc == LOVE_OK) brc = cuda_check(cudaStreamSynchronize(st[0]));
    if (brc != LOVE_OK) {
      free_q();
      cudaStreamSynchronize(st[0]);
      if (brc != LOVE_ERR_UNSUPPORTED) {
        cudaEventDestroy(fork);
        return brc;
      }
      batched = false;   // a GP of a form the batched run does not take: per-GP runs
    }
  }
  std::atomic<int> next{0};
  auto work = [&](int w) {
    cudaSetDevice(dev);
    // this worker's work buffers (and its mean-solve threads') are reused from GP to GP
    ScratchCache own, mean;
    thread_scratch() = &own;
    thread_mean_scratch() = &mean;
    struct Uninstall {
      ~Uninstall() {
        thread_scratch() = nullptr;
        thread_mean_scratch() = nullptr;
      }
    } uninstall;
    for (;;) {
      const int b = next.fetch_add(1);
      if (b >= B) break;
      if (batched) {
        float* q = Qb[b];
        Qb[b] = nullptr;   // owned by the call from here on
        rc[b] = precompute_from_lanczos(skis[b], opts, st[w], q, bl.gp[b], bl.rows, bl.ms, &caches[b], &ke[b]);
      } else {
        rc[b] = love_precompute(skis[b], opts, (love_stream_t)st[w], &caches[b], &ke[b]);
      }
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w) {
    try {
      th.emplace_back(work, w);
    } catch (...) {   // no more host threads: the started workers take the rest
      break;
    }
  }
  work(0);
  for (auto& t : th) t.join();
  cudaEventDestroy(fork);
  love_status first = LOVE_OK;
  for (int b = 0; b < B; ++b)
    if (rc[b] != LOVE_OK) {
      first = rc[b];
      break;
    }
  if (first != LOVE_OK) {
    for (int b = 0; b < B; ++b) {
      if (caches[b]) love_cache_destroy(caches[b]);
      caches[b] = nullptr;
    }
    return first;
  }
  if (k_eff)
    for (int b = 0; b < B; ++b) k_eff[b] = ke[b];
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_batch_create(int B, const love_cache_t* caches, const int64_t* t_off, love_stream_t stream,
                              love_batch_t* out) try {
  if (!out) return LOVE_ERR_ARG;
  *out = nullptr;
  if (B < 1 || !caches || !t_off || t_off[0] != 0) return LOVE_ERR_ARG;
  for (int b = 0; b < B; ++b) {
    if (!caches[b] || t_off[b + 1] < t_off[b]) return LOVE_ERR_ARG;
    if (caches[b]->grid.dim != caches[0]->grid.dim || caches[b]->dtype != caches[0]->dtype ||
        caches[b]->cache_dtype != caches[0]->cache_dtype)
      return LOVE_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  love_batch* bt = new love_batch();
  bt->B = B;
  bt->dim = caches[0]->grid.dim;
  bt->dtype = caches[0]->dtype;
  bt->cache_dtype = caches[0]->cache_dtype;
  bt->caches.assign(caches, caches + B);
  bt->t_off.assign(t_off, t_off + B + 1);
  bt->alloc = caches[0]->alloc;
  bt->desc_bytes = predict_desc_bytes();
  std::vector<unsigned char> hd(bt->desc_bytes * B);
  for (int b = 0; b < B; ++b) predict_fill_desc(caches[b], hd.data() + bt->desc_bytes * b);
  std::vector<PredChunk> ch;
  for (int b = 0; b < B; ++b) {
    const int64_t t = t_off[b + 1] - t_off[b];
    for (int64_t r = 0; r < t; r += kChunkRows) ch.push_back(PredChunk{b, 0, r, std::min(t, r + kChunkRows)});
  }
  if (ch.size() > (size_t)0x7fffffff) {
    delete bt;
    return LOVE_ERR_ARG;
  }
  bt->nchunks = (int)ch.size();
  bt->d_desc = bt->alloc.alloc(bt->desc_bytes * B, s);
  bt->d_toff = (int64_t*)bt->alloc.alloc(sizeof(int64_t) * (B + 1), s);
  bt->d_chunks = (PredChunk*)bt->alloc.alloc(sizeof(PredChunk) * std::max(bt->nchunks, 1), s);
  love_status rc = (bt->d_desc && bt->d_toff && bt->d_chunks) ? LOVE_OK : LOVE_ERR_OOM;
  if (rc == LOVE_OK)
    rc = cuda_check(cudaMemcpyAsync(bt->d_desc, hd.data(), hd.size(), cudaMemcpyHostToDevice, s));
  if (rc == LOVE_OK)
    rc = cuda_check(cudaMemcpyAsync(bt->d_toff, t_off, sizeof(int64_t) * (B + 1), cudaMemcpyHostToDevice, s));
  if (rc == LOVE_OK && bt->nchunks)
    rc = cuda_check(
        cudaMemcpyAsync(bt->d_chunks, ch.data(), sizeof(PredChunk) * ch.size(), cudaMemcpyHostToDevice, s));
  if (rc == LOVE_OK) rc = cuda_check(cudaStreamSynchronize(s));
  if (rc == LOVE_OK) rc = autotune(bt, s);
  if (rc != LOVE_OK) {
    batch_free(bt, s);
    return rc;
  }
  *out = bt;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_batch_destroy(love_batch_t b) try {
  if (!b) return LOVE_ERR_ARG;
  batch_free(b, 0);
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

love_status love_predict_batched(love_batch_t b, const void* x, void* mean, void* var, love_stream_t stream) try {
  if (!b) return LOVE_ERR_ARG;
  if (b->t_off[b->B] == 0) return LOVE_OK;
  if (!x || !var) return LOVE_ERR_ARG;
  if (mean)
    for (auto* c : b->caches)
      if (!(c->flags & LOVE_WANT_MEAN)) return LOVE_ERR_STATE;
  return batch_predict(b, x, mean, var, b->lanes, b->ctas, (cudaStream_t)stream);
}
LOVE_ENTRY_CATCH

love_status love_sample_batched(love_batch_t b, const void* x, int s_count, uint64_t seed, void* out,
                                love_stream_t stream) try {
  if (!b || s_count < 0) return LOVE_ERR_ARG;
  if (s_count == 0 || b->t_off[b->B] == 0) return LOVE_OK;
  if (!x || !out) return LOVE_ERR_ARG;
  for (auto* c : b->caches)
    if (!(c->flags & LOVE_WANT_SAMPLER) || !c->S) return LOVE_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  LOVE_TRY(ensure_ws(b, s_count, s));
  return batch_sample(b, x, s_count, seed, out, s);
}
LOVE_ENTRY_CATCH

love_status love_batch_serve(love_batch_t b, const void* x, void* mean, void* var, int s_count, uint64_t seed,
                             void* samples, int use_graph, love_stream_t stream) try {
  if (!b || s_count < 0 || (s_count > 0 && !samples)) return LOVE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (!use_graph) {
    LOVE_TRY(love_predict_batched(b, x, mean, var, stream));
    return s_count ? love_sample_batched(b, x, s_count, seed, samples, stream) : LOVE_OK;
  }
  if (!b->gstream) {
    LOVE_CUDA(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking));
    LOVE_CUDA(cudaEventCreateWithFlags(&b->gev_in, cudaEventDisableTiming));
    LOVE_CUDA(cudaEventCreateWithFlags(&b->gev_out, cudaEventDisableTiming));
  }
  const bool hit = b->gexec && b->gx == x && b->gmean == mean && b->gvar == var && b->gs == s_count &&
                   b->gseed == seed && b->gsamples == samples;
  if (!hit) {
    // first time for these arguments: one eager call (argument checks, work
    // space), then capture the same launches on the graph stream
    LOVE_TRY(love_predict_batched(b, x, mean, var, stream));
    if (s_count) LOVE_TRY(love_sample_batched(b, x, s_count, seed, samples, stream));
    LOVE_CUDA(cudaStreamSynchronize(s));
    if (b->t_off[b->B] == 0) return LOVE_OK;
    LOVE_CUDA(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeRelaxed));
    love_status rc = LOVE_OK;
    try {   // whatever happens, the capture is ended below
      rc = batch_predict(b, x, mean, var, b->lanes, b->ctas, b->gstream);
      if (rc == LOVE_OK && s_count) rc = batch_sample(b, x, s_count, seed, samples, b->gstream);
    } catch (...) {
      rc = LOVE_ERR_OOM;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->gstream, &graph);
    if (rc == LOVE_OK && e != cudaSuccess) rc = cuda_check(e);
    cudaGraphExec_t ex = nullptr;
    if (rc == LOVE_OK) rc = cuda_check(cudaGraphInstantiate(&ex, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    if (rc != LOVE_OK) return rc;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->gexec = ex;
    ++b->gcaptures;
    b->gx = x;
    b->gmean = mean;
    b->gvar = var;
    b->gs = s_count;
    b->gseed = seed;
    b->gsamples = samples;
    return LOVE_OK;
  }
  // replay on the graph stream, ordered after and joined back into the caller's stream
  LOVE_CUDA(cudaEventRecord(b->gev_in, s));
  LOVE_CUDA(cudaStreamWaitEvent(b->gstream, b->gev_in, 0));
  LOVE_CUDA(cudaGraphLaunch(b->gexec, b->gstream));
  LOVE_CUDA(cudaEventRecord(b->gev_out, b->gstream));
  return cuda_check(cudaStreamWaitEvent(s, b->gev_out, 0));
}
LOVE_ENTRY_CATCH

love_status love_batch_info(love_batch_t b, love_batch_info_t* info) try {
  if (!b || !info) return LOVE_ERR_ARG;
  std::memset(info, 0, sizeof(*info));
  info->lanes_per_point = b->lanes;
  info->ctas_per_sm = b->ctas;
  info->n_candidates = b->n_cand;
  for (int i = 0; i < b->n_cand && i < 16; ++i) info->candidate_ms[i] = b->cand_ms[i];
  info->chunks = b->nchunks;
  info->graph_captures = b->gcaptures;
  info->graph_captures_dropped = b->gcaptures_dropped;
  return LOVE_OK;
}
LOVE_ENTRY_CATCH

}  // extern "C"
