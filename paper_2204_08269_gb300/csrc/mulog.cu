// mu-log compression of scattering paths (Sec. 4.3, Eq. 6-7), on CUDA cores.
//
//   k_mulog_mean : mu[p] = (1/B) sum_b sum_m S[b][p][m]  (one block per path, FP64 sums in a
//                  fixed order)
//   k_mulog      : out = log(1 + S / (eps mu[p]))
//   k_mulog_bwd  : g_S = g_out / (eps mu[p] + S)
// S is any [B][P][M] array: the S2 paths of the transform (M = n_lam_out n_t), the time
// scattering paths (M = n_t), S1 rows, ...
#include <algorithm>

#include "internal.h"

namespace jtfs {
namespace {

constexpr int kMlThreads = 256;

__global__ void k_mulog_mean(const float* __restrict__ s, long long B, long long P, long long M,
                             float* __restrict__ mu) {
  __shared__ double red[kMlThreads / 32];
  const long long p = blockIdx.x;
  double acc = 0.0;
  for (long long b = 0; b < B; ++b) {
    const float* row = s + (b * P + p) * M;
    for (long long m = threadIdx.x; m < M; m += blockDim.x) acc += (double)row[m];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kMlThreads / 32; ++w) t += red[w];
    mu[p] = (float)(t / (double)B);
  }
}

__global__ void k_mulog(const float* __restrict__ s, long long total, long long P, long long M,
                        const float* __restrict__ mu, float eps, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = (i / M) % P;
    out[i] = log1pf(s[i] / (eps * __ldg(&mu[p])));
  }
}

__global__ void k_mulog_bwd(const float* __restrict__ s, long long total, long long P,
                            long long M, const float* __restrict__ mu, float eps,
                            const float* __restrict__ g, float* __restrict__ gs) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long p = (i / M) % P;
    gs[i] = g[i] / (eps * __ldg(&mu[p]) + s[i]);
  }
}

bool bad_sizes(const void* a, const void* b, int64_t B, int64_t P, int64_t M) {
  if (!a || !b || B < 0 || P < 1 || M < 1 || B > (1LL << 24) || P > (1LL << 24) ||
      M > (1LL << 30)) {
    set_error("bad pointer or size");
    return true;
  }
  return false;
}

int grid_for(long long total) {
  return (int)std::min<long long>(152LL * 8, (total + kMlThreads - 1) / kMlThreads);
}

}  // namespace
}  // namespace jtfs

using namespace jtfs;

extern "C" {

jtfs_status jtfs_mulog_mean(const float* s, int64_t B, int64_t P, int64_t M, float* mu,
                            void* stream) {
  if (bad_sizes(s, mu, B, P, M) || B < 1) {
    if (B < 1) set_error("the mean needs at least one example");
    return JTFS_ERR_INVALID_ARG;
  }
  k_mulog_mean<<<(unsigned)P, kMlThreads, 0, (cudaStream_t)stream>>>(s, B, P, M, mu);
  return cuda_check(cudaGetLastError(), "k_mulog_mean");
}

jtfs_status jtfs_mulog(const float* s, int64_t B, int64_t P, int64_t M, const float* mu,
                       float eps, float* out, void* stream) {
  if (bad_sizes(s, out, B, P, M) || !mu || !(eps > 0.f)) {
    if (!mu || !(eps > 0.f)) set_error("NULL mu or eps <= 0");
    return JTFS_ERR_INVALID_ARG;
  }
  const long long total = (long long)B * P * M;
  if (total == 0) return JTFS_OK;
  k_mulog<<<grid_for(total), kMlThreads, 0, (cudaStream_t)stream>>>(s, total, P, M, mu, eps, out);
  return cuda_check(cudaGetLastError(), "k_mulog");
}

jtfs_status jtfs_mulog_backward(const float* s, int64_t B, int64_t P, int64_t M,
                                const float* mu, float eps, const float* g_out, float* g_s,
                                void* stream) {
  if (bad_sizes(s, g_s, B, P, M) || !mu || !g_out || !(eps > 0.f)) {
    if (!mu || !g_out || !(eps > 0.f)) set_error("NULL mu / g_out or eps <= 0");
    return JTFS_ERR_INVALID_ARG;
  }
  const long long total = (long long)B * P * M;
  if (total == 0) return JTFS_OK;
  k_mulog_bwd<<<grid_for(total), kMlThreads, 0, (cudaStream_t)stream>>>(s, total, P, M, mu, eps,
                                                                        g_out, g_s);
  return cuda_check(cudaGetLastError(), "k_mulog_bwd");
}

}  // extern "C"
