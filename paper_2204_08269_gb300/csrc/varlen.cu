// Uneven-length batches.  The paper transforms one length at a time; a batch of signals of
// different lengths is handled here by zero-padding each signal to
//     N_i = max(2^ceil(log2 len_i), 2^(J+3))
// (a power of two, as the periodic transform needs, and long enough for the coarsest
// first-order filter), transforming it with the plan of that length and keeping the first
// ceil(len_i / T) frames of S0, S1 and S2.  Signals of the same N_i form one bucket, run in
// sub-batches through jtfs_forward_backward; small kernels gather the packed input and
// cotangents into the padded batch and scatter outputs and g_x back.  The whole step can be
// captured into one CUDA graph and replayed.
#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "internal.h"

namespace jtfs {
namespace {

// xb[b][n] = n < len_b ? xp[off_b + n] : 0
__global__ void k_vl_gather_x(const float* __restrict__ xp, const long long* __restrict__ off,
                              const int* __restrict__ len, int N, float* __restrict__ xb) {
  const int b = blockIdx.y;
  const long long o = off[b];
  const int L = len[b];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
    xb[(size_t)b * N + n] = n < L ? xp[o + n] : 0.f;
}

// xp[off_b + n] = xb[b][n] for n < len_b
__global__ void k_vl_scatter_x(const float* __restrict__ xb, const long long* __restrict__ off,
                               const int* __restrict__ len, int N, float* __restrict__ xp) {
  const int b = blockIdx.y;
  const long long o = off[b];
  const int L = len[b];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < L; n += gridDim.x * blockDim.x)
    xp[o + n] = xb[(size_t)b * N + n];
}

// Frame-major rows: batch [b][r][t < n_t] <-> packed [off_b + r * fr_b + t] for t < fr_b.
// TO_PACKED = 1 copies batch -> packed; 0 copies packed -> batch (zero beyond fr_b, and zero
// everywhere when the packed pointer is NULL).
template <int TO_PACKED>
__global__ void k_vl_frames(const float* __restrict__ src, float* __restrict__ dst,
                            const long long* __restrict__ off, const int* __restrict__ fr,
                            int rows, int n_t) {
  const int b = blockIdx.y;
  const long long o = off[b];
  const int F = fr[b];
  const long long total = (long long)rows * n_t;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n_t), t = (int)(i % n_t);
    const size_t bi = (size_t)b * total + i;
    if (TO_PACKED) {
      if (t < F) dst[o + (long long)r * F + t] = src[bi];
    } else {
      dst[bi] = (src && t < F) ? src[o + (long long)r * F + t] : 0.f;
    }
  }
}

}  // namespace
}  // namespace jtfs

using namespace jtfs;

struct jtfs_varlen {
  jtfs_config cfg;
  int64_t B = 0;
  int device = 0;
  std::vector<int64_t> len;
  std::vector<int64_t> x_off, s0_off, s1_off, s2_off;   // B + 1 entries each
  struct Chunk {           // one sub-batch of one bucket
    jtfs_plan* plan;       // shared by the chunks of a bucket (owned by the bucket)
    int count;
    long long* d_xoff;     // [count] into the packed x / g_x
    int* d_len;
    long long* d_s0off;
    long long* d_s1off;
    long long* d_s2off;
    int* d_frames;
  };
  std::vector<jtfs_plan*> plans;
  std::vector<std::pair<jtfs_plan*, std::vector<int>>> buckets;   // plan, signals (in order)
  std::vector<int> frames;
  std::vector<Chunk> chunks;
  void* d_meta = nullptr;
  size_t ws_bytes = 0;     // the current chunks': plan workspace + padded batch buffers
  size_t ws_cap = 0;       // the workspace the caller sizes: that of chunks of chunk_max
  int chunk_max = 64;      // sub-batch size given at creation (the largest one tried)
  int chunk = 64;          // sub-batch size in use
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int64_t vl_pad(const jtfs_config& c, int64_t len) {
  int64_t n = 1;
  while (n < len) n <<= 1;
  return std::max<int64_t>(n, (int64_t)1 << (c.J + 3));
}

// bytes of the padded batch buffers of one chunk (x, s0, s1, s2, u1, g_s0, g_s1, g_s2, g_x)
size_t vl_batch_bytes(const jtfs_plan* p, int cnt) {
  jtfs_shapes sh;
  jtfs_plan_shapes(p, &sh);
  auto a = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t c = (size_t)cnt;
  return 2 * a(c * sh.N * 4) + 2 * a(c * sh.s0_len * 4) + 2 * a(c * sh.s1_len * 4) +
         2 * a(c * sh.s2_len * 4) + a(c * sh.u1_len * 4);
}

jtfs_status vl_run(const jtfs_varlen* v, const float* x, const float* gs0, const float* gs1,
                   const float* gs2, float* s0, float* s1, float* s2, float* gx, void* ws,
                   size_t ws_bytes, cudaStream_t st) {
  if (!ws || ws_bytes < v->ws_bytes) {
    set_error("varlen workspace needs " + std::to_string(v->ws_bytes) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  jtfs_status rc;
  for (const auto& ch : v->chunks) {
    jtfs_shapes sh;
    jtfs_plan_shapes(ch.plan, &sh);
    const int cnt = ch.count;
    const int N = (int)sh.N, nt = (int)sh.n_t;
    char* base = (char*)ws;
    size_t off = 0;
    auto take = [&](size_t bytes) { char* q = base + off; off += (bytes + 255) & ~(size_t)255; return q; };
    float* xb = (float*)take((size_t)cnt * N * 4);
    float* gxb = (float*)take((size_t)cnt * N * 4);
    float* s0b = (float*)take((size_t)cnt * sh.s0_len * 4);
    float* g0b = (float*)take((size_t)cnt * sh.s0_len * 4);
    float* s1b = (float*)take((size_t)cnt * sh.s1_len * 4);
    float* g1b = (float*)take((size_t)cnt * sh.s1_len * 4);
    float* s2b = (float*)take((size_t)cnt * sh.s2_len * 4);
    float* g2b = (float*)take((size_t)cnt * sh.s2_len * 4);
    float* u1b = (float*)take((size_t)cnt * sh.u1_len * 4);
    void* pws = base + off;
    const size_t pws_bytes = ws_bytes - off;
    const dim3 gx_grid((unsigned)std::min<int64_t>((N + 255) / 256, 1024), (unsigned)cnt);
    k_vl_gather_x<<<gx_grid, 256, 0, st>>>(x, ch.d_xoff, ch.d_len, N, xb);
    const int rows1 = (int)sh.n1, rows2 = (int)(sh.s2_paths * sh.n_lam_out);
    auto grid_for = [&](int rows) {
      return dim3((unsigned)std::min<int64_t>(((int64_t)rows * nt + 255) / 256, 1024), (unsigned)cnt);
    };
    k_vl_frames<0><<<grid_for(1), 256, 0, st>>>(gs0, g0b, ch.d_s0off, ch.d_frames, 1, nt);
    k_vl_frames<0><<<grid_for(rows1), 256, 0, st>>>(gs1, g1b, ch.d_s1off, ch.d_frames, rows1, nt);
    k_vl_frames<0><<<grid_for(rows2), 256, 0, st>>>(gs2, g2b, ch.d_s2off, ch.d_frames, rows2, nt);
    if ((rc = cuda_check(cudaGetLastError(), "varlen gather")) != JTFS_OK) return rc;
    if ((rc = jtfs_forward_backward(ch.plan, xb, cnt, g0b, g1b, g2b, s0b, s1b, s2b, u1b, gxb, pws,
                                    pws_bytes, st)) != JTFS_OK)
      return rc;
    k_vl_frames<1><<<grid_for(1), 256, 0, st>>>(s0b, s0, ch.d_s0off, ch.d_frames, 1, nt);
    k_vl_frames<1><<<grid_for(rows1), 256, 0, st>>>(s1b, s1, ch.d_s1off, ch.d_frames, rows1, nt);
    k_vl_frames<1><<<grid_for(rows2), 256, 0, st>>>(s2b, s2, ch.d_s2off, ch.d_frames, rows2, nt);
    k_vl_scatter_x<<<gx_grid, 256, 0, st>>>(gxb, ch.d_xoff, ch.d_len, N, gx);
    if ((rc = cuda_check(cudaGetLastError(), "varlen scatter")) != JTFS_OK) return rc;
  }
  return JTFS_OK;
}

// Splits every bucket into sub-batches of at most `chunk` signals and uploads their index
// tables (per sub-batch [xoff][s0off][s1off][s2off] as int64, then [len][frames] as int32),
// replacing earlier ones; sets ws_bytes for them.
jtfs_status vl_build_chunks(jtfs_varlen* v, int chunk) {
  if (v->d_meta) { cudaFree(v->d_meta); v->d_meta = nullptr; }
  v->chunks.clear();
  v->ws_bytes = 0;
  v->chunk = chunk;
  struct Pending { jtfs_plan* plan; std::vector<int> idx; };
  std::vector<Pending> pend;
  for (auto& bk : v->buckets) {
    const auto& ids = bk.second;
    for (size_t s = 0; s < ids.size(); s += (size_t)chunk) {
      Pending pc;
      pc.plan = bk.first;
      pc.idx.assign(ids.begin() + s, ids.begin() + std::min(ids.size(), s + (size_t)chunk));
      pend.push_back(pc);
    }
  }
  std::vector<char> host;
  std::vector<size_t> at;
  for (auto& pc : pend) {
    const size_t n = pc.idx.size();
    at.push_back(host.size());
    const size_t bytes = ((n * 8 * 4 + n * 4 * 2) + 255) & ~(size_t)255;
    const size_t o = host.size();
    host.resize(o + bytes, 0);
    long long* L64 = (long long*)(host.data() + o);
    int* L32 = (int*)(host.data() + o + n * 8 * 4);
    for (size_t k = 0; k < n; ++k) {
      const int i = pc.idx[k];
      L64[k] = v->x_off[i];
      L64[n + k] = v->s0_off[i];
      L64[2 * n + k] = v->s1_off[i];
      L64[3 * n + k] = v->s2_off[i];
      L32[k] = (int)v->len[i];
      L32[n + k] = v->frames[i];
    }
  }
  jtfs_status rc;
  if ((rc = cuda_check(cudaMalloc(&v->d_meta, std::max<size_t>(256, host.size())), "varlen tables")) != JTFS_OK ||
      (rc = cuda_check(cudaMemcpy(v->d_meta, host.data(), host.size(), cudaMemcpyHostToDevice), "varlen upload")) != JTFS_OK)
    return rc;
  for (size_t c = 0; c < pend.size(); ++c) {
    const size_t n = pend[c].idx.size();
    char* base = (char*)v->d_meta + at[c];
    jtfs_varlen::Chunk ch;
    ch.plan = pend[c].plan;
    ch.count = (int)n;
    ch.d_xoff = (long long*)base;
    ch.d_s0off = ch.d_xoff + n;
    ch.d_s1off = ch.d_xoff + 2 * n;
    ch.d_s2off = ch.d_xoff + 3 * n;
    ch.d_len = (int*)(base + n * 8 * 4);
    ch.d_frames = ch.d_len + n;
    v->chunks.push_back(ch);
    size_t pws = 0;
    jtfs_workspace_bytes(ch.plan, (int64_t)n, 1, &pws);
    v->ws_bytes = std::max(v->ws_bytes, vl_batch_bytes(ch.plan, (int)n) + pws);
  }
  return JTFS_OK;
}

}  // namespace

extern "C" {

int64_t jtfs_varlen_padded_length(const jtfs_config* cfg, int64_t len) {
  if (!cfg || len < 1 || cfg->J < 0 || cfg->J > 40) return 0;
  return vl_pad(*cfg, len);
}

jtfs_status jtfs_varlen_create(const jtfs_config* cfg, const int64_t* len, int64_t B,
                               int32_t chunk, jtfs_varlen** out) {
  if (!cfg || !len || !out || B < 1 || B > (1 << 20) || chunk < 0) {
    set_error("bad argument");
    return JTFS_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (cfg->out_3d != 1) {
    set_error("uneven-length batches keep their own packed layouts: out_3d must be 1");
    return JTFS_ERR_INVALID_ARG;
  }
  for (int64_t i = 0; i < B; ++i)
    if (len[i] < 1 || len[i] > ((int64_t)1 << 24)) {
      set_error("signal length out of range [1, 2^24]");
      return JTFS_ERR_INVALID_ARG;
    }
  auto* v = new jtfs_varlen();
  v->cfg = *cfg;
  v->B = B;
  v->len.assign(len, len + B);
  if (chunk > 0) v->chunk_max = chunk;
  cudaGetDevice(&v->device);
  // buckets by padded length, in signal order within a bucket
  std::map<int64_t, std::vector<int>> buckets;
  for (int64_t i = 0; i < B; ++i) buckets[vl_pad(*cfg, len[i])].push_back((int)i);
  jtfs_status rc = JTFS_OK;
  std::map<int64_t, jtfs_plan*> plan_of;
  for (auto& kv : buckets) {
    jtfs_plan* p = nullptr;
    if ((rc = jtfs_plan_create(cfg, kv.first, &p)) != JTFS_OK) {
      jtfs_varlen_destroy(v);
      return rc;
    }
    v->plans.push_back(p);
    plan_of[kv.first] = p;
  }
  // packed offsets in signal order
  v->x_off.assign(B + 1, 0);
  v->s0_off.assign(B + 1, 0);
  v->s1_off.assign(B + 1, 0);
  v->s2_off.assign(B + 1, 0);
  std::vector<int> frames(B);
  for (int64_t i = 0; i < B; ++i) {
    jtfs_shapes sh;
    jtfs_plan_shapes(plan_of[vl_pad(*cfg, len[i])], &sh);
    frames[i] = (int)((len[i] + cfg->T - 1) / cfg->T);
    v->x_off[i + 1] = v->x_off[i] + len[i];
    v->s0_off[i + 1] = v->s0_off[i] + frames[i];
    v->s1_off[i + 1] = v->s1_off[i] + sh.n1 * frames[i];
    v->s2_off[i + 1] = v->s2_off[i] + sh.s2_paths * sh.n_lam_out * frames[i];
  }
  v->frames = frames;
  for (auto& kv : buckets) v->buckets.push_back({plan_of[kv.first], kv.second});
  if ((rc = vl_build_chunks(v, v->chunk_max)) != JTFS_OK) {
    jtfs_varlen_destroy(v);
    return rc;
  }
  v->ws_cap = v->ws_bytes;
  *out = v;
  return JTFS_OK;
}

void jtfs_varlen_destroy(jtfs_varlen* v) {
  if (!v) return;
  if (v->exec) cudaGraphExecDestroy(v->exec);
  if (v->graph) cudaGraphDestroy(v->graph);
  if (v->d_meta) cudaFree(v->d_meta);
  for (jtfs_plan* p : v->plans) jtfs_plan_destroy(p);
  delete v;
}

jtfs_status jtfs_varlen_layout(const jtfs_varlen* v, int64_t* x_off, int64_t* s0_off,
                               int64_t* s1_off, int64_t* s2_off) {
  if (!v) { set_error("NULL varlen"); return JTFS_ERR_INVALID_ARG; }
  const size_t n = (size_t)v->B + 1;
  if (x_off) std::copy(v->x_off.begin(), v->x_off.begin() + n, x_off);
  if (s0_off) std::copy(v->s0_off.begin(), v->s0_off.begin() + n, s0_off);
  if (s1_off) std::copy(v->s1_off.begin(), v->s1_off.begin() + n, s1_off);
  if (s2_off) std::copy(v->s2_off.begin(), v->s2_off.begin() + n, s2_off);
  return JTFS_OK;
}

jtfs_status jtfs_varlen_workspace_bytes(const jtfs_varlen* v, size_t* out) {
  if (!v || !out) { set_error("bad argument"); return JTFS_ERR_INVALID_ARG; }
  *out = v->ws_cap;
  return JTFS_OK;
}

jtfs_status jtfs_varlen_tune_schedule(jtfs_varlen* v, const float* x, const float* g_s0,
                                      const float* g_s1, const float* g_s2, float* s0,
                                      float* s1, float* s2, float* g_x, void* ws,
                                      size_t ws_bytes, void* stream, int32_t* chosen) {
  if (!v || !x || !s0 || !s1 || !s2 || !g_x) { set_error("NULL argument"); return JTFS_ERR_INVALID_ARG; }
  if (!ws || ws_bytes < v->ws_cap) {
    set_error("varlen workspace needs " + std::to_string(v->ws_cap) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int> cand;
  for (int c = 16; c < v->chunk_max; c <<= 1) cand.push_back(c);
  cand.push_back(v->chunk_max);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  jtfs_status rc = cuda_check(cudaEventCreate(&e0), "event");
  if (rc == JTFS_OK) rc = cuda_check(cudaEventCreate(&e1), "event");
  int best = v->chunk;
  float best_ms = 0.f;
  for (size_t i = 0; i < cand.size() && rc == JTFS_OK; ++i) {
    if ((rc = vl_build_chunks(v, cand[i])) != JTFS_OK) break;
    // one untimed pass (first launches, attributes), then two timed ones
    if ((rc = vl_run(v, x, g_s0, g_s1, g_s2, s0, s1, s2, g_x, ws, ws_bytes, st)) != JTFS_OK) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 2 && rc == JTFS_OK; ++r)
      rc = vl_run(v, x, g_s0, g_s1, g_s2, s0, s1, s2, g_x, ws, ws_bytes, st);
    cudaEventRecord(e1, st);
    if (rc == JTFS_OK) rc = cuda_check(cudaEventSynchronize(e1), "tune sync");
    float ms = 0.f;
    if (rc == JTFS_OK) rc = cuda_check(cudaEventElapsedTime(&ms, e0, e1), "tune time");
    if (rc == JTFS_OK && (i == 0 || ms < best_ms)) { best_ms = ms; best = cand[i]; }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // a captured graph holds the old sub-batches: drop it (capture again after tuning)
  if (v->exec) { cudaGraphExecDestroy(v->exec); v->exec = nullptr; }
  if (v->graph) { cudaGraphDestroy(v->graph); v->graph = nullptr; }
  jtfs_status rb = vl_build_chunks(v, best);
  if (rc != JTFS_OK) return rc;
  if (rb != JTFS_OK) return rb;
  if (chosen) chosen[0] = best;
  return JTFS_OK;
}

jtfs_status jtfs_varlen_forward_backward(const jtfs_varlen* v, const float* x, const float* g_s0,
                                         const float* g_s1, const float* g_s2, float* s0,
                                         float* s1, float* s2, float* g_x, void* ws,
                                         size_t ws_bytes, void* stream) {
  if (!v || !x || !s0 || !s1 || !s2 || !g_x) { set_error("NULL argument"); return JTFS_ERR_INVALID_ARG; }
  return vl_run(v, x, g_s0, g_s1, g_s2, s0, s1, s2, g_x, ws, ws_bytes, (cudaStream_t)stream);
}

jtfs_status jtfs_varlen_capture(jtfs_varlen* v, const float* x, const float* g_s0,
                                const float* g_s1, const float* g_s2, float* s0, float* s1,
                                float* s2, float* g_x, void* ws, size_t ws_bytes, void* stream) {
  if (!v || !x || !s0 || !s1 || !s2 || !g_x || !stream) {
    set_error("NULL argument (capture needs a non-default stream)");
    return JTFS_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  jtfs_status rc;
  // one uncaptured pass sets every kernel attribute the launches need
  if ((rc = vl_run(v, x, g_s0, g_s1, g_s2, s0, s1, s2, g_x, ws, ws_bytes, st)) != JTFS_OK) return rc;
  if ((rc = cuda_check(cudaStreamSynchronize(st), "varlen warm-up")) != JTFS_OK) return rc;
  if (v->exec) { cudaGraphExecDestroy(v->exec); v->exec = nullptr; }
  if (v->graph) { cudaGraphDestroy(v->graph); v->graph = nullptr; }
  if ((rc = cuda_check(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed), "begin capture")) != JTFS_OK) return rc;
  jtfs_status run = vl_run(v, x, g_s0, g_s1, g_s2, s0, s1, s2, g_x, ws, ws_bytes, st);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(st, &g);
  if (run != JTFS_OK) {
    if (g) cudaGraphDestroy(g);
    return run;
  }
  if ((rc = cuda_check(e, "end capture")) != JTFS_OK) return rc;
  v->graph = g;
  return cuda_check(cudaGraphInstantiate(&v->exec, g, 0), "graph instantiate");
}

jtfs_status jtfs_varlen_autotune(jtfs_varlen* v, void* ws, size_t ws_bytes, void* stream) {
  if (!v) { set_error("NULL varlen"); return JTFS_ERR_INVALID_ARG; }
  if (!ws || ws_bytes < v->ws_bytes) {
    set_error("varlen workspace needs " + std::to_string(v->ws_bytes) + " bytes");
    return JTFS_ERR_WORKSPACE;
  }
  for (jtfs_plan* p : v->plans) {
    int most = 0;
    for (const auto& ch : v->chunks)
      if (ch.plan == p) most = std::max(most, ch.count);
    if (most == 0) continue;
    jtfs_status rc = jtfs_plan_autotune(p, most, ws, ws_bytes, stream, nullptr);
    if (rc != JTFS_OK) return rc;
  }
  return JTFS_OK;
}

jtfs_status jtfs_varlen_replay(const jtfs_varlen* v, void* stream) {
  if (!v || !v->exec) { set_error("no captured graph"); return JTFS_ERR_INVALID_ARG; }
  return cuda_check(cudaGraphLaunch(v->exec, (cudaStream_t)stream), "graph launch");
}

}  // extern "C"
