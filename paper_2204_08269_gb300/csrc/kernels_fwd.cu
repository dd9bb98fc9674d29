// Forward JTFS kernels (Sec. 2, Eq. 2-4) on CUDA cores, FP32.
//
//   k_xfft_sub / k_xfft_combine : x-hat[k] for 0 <= k < N/2 (decimated length-N FFT)
//   k_s0                        : S0[t] = sum_n phi_T[(tT - n) mod N] x[n] (compensated sum)
//   k_scalogram                 : per (lambda, signal): periodise x-hat * psi-hat_lambda to
//                                 L_lambda bins, inverse FFT, modulus -> U1 row (checkpoint),
//                                 FFT of the row -> U1-hat, S1 row (the Riemann sum of
//                                 phi_T, evaluated on the row spectrum)
//   k_second_order_rows         : per (alpha, block of lambda' rows, signal): U1-hat *
//                                 psi-hat_alpha folded to L_alpha bins, batched inverse FFT
//                                 -> Y_alpha rows
//   k_joint_fwd_simt            : per (c, alpha, signal): Z = W_c Y_alpha (zero-padded
//                                 convolution along lambda), |Z|, phi_T then phi_F pooling -> S2
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "stages.cuh"
#include "umma.cuh"

namespace jtfs {
namespace {

namespace cg = cooperative_groups;

// S0[t] = sum_n phi_T[(tT - n) mod N] x[n], in the time domain from x itself, to about FP64
// accuracy.  For band-pass inputs S0 is a small difference of large terms: for click trains
// through resonators |S0| is about 2e-6 of sum |phi_T x|, below the rounding of FP32 weights
// and products.  So every term is formed exactly in two FP32 parts, phi_T = hi + lo and
// hi x = p + e (e from an FMA), and summed with a Neumaier (sum, correction) pair per thread;
// the pairs are added in FP64.  The spectral form from x-hat would inherit the FP32 FFT's
// rounding, which is of the size of S0 itself for such inputs.
// One cluster of kS0Split CTAs per (frame, signal): CTA r sums the r-th slice of the samples
// (weights and samples both read contiguously) and hands its FP64 partial to CTA 0 through
// distributed shared memory, which adds them in a fixed order.
constexpr int kS0Split = 8, kS0Threads = 256;

__global__ void __cluster_dims__(kS0Split, 1, 1) __launch_bounds__(kS0Threads)
k_s0(DevPlan P, const float* __restrict__ x, float* __restrict__ s0) {
  __shared__ double red[kS0Threads / 32];
  __shared__ double parts[kS0Split];
  cg::cluster_group cl = cg::this_cluster();
  const int part = (int)cl.block_rank(), t = blockIdx.x / kS0Split, b = blockIdx.y;
  const int chunk = P.N / kS0Split;
  const float* xb = x + (size_t)b * P.N;
  const long long tT = (long long)t * P.T;
  float sum = 0.f, cor = 0.f;
  for (int n = part * chunk + threadIdx.x; n < (part + 1) * chunk; n += blockDim.x) {
    const int k = (int)((tT - n) & (P.N - 1));
    const float v = xb[n], hi = __ldg(&P.phiT[k]), lo = __ldg(&P.phiT_lo[k]);
    const float pr = __fmul_rn(hi, v);
    const float e = fmaf(lo, v, fmaf(hi, v, -pr));
    const float u = __fadd_rn(sum, pr);
    const float d = fabsf(sum) >= fabsf(pr) ? __fadd_rn(__fsub_rn(sum, u), pr)
                                            : __fadd_rn(__fsub_rn(pr, u), sum);
    cor = __fadd_rn(cor, __fadd_rn(d, e));
    sum = u;
  }
  double acc = (double)sum + (double)cor;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < kS0Threads / 32; ++i) v += red[i];
    cl.map_shared_rank(parts, 0)[part] = v;
  }
  cl.sync();
  if (part == 0 && threadIdx.x == 0) {
    double v = 0.0;
    for (int r = 0; r < kS0Split; ++r) v += parts[r];
    s0[(size_t)b * P.n_t + t] = (float)v;
  }
}

__global__ void __launch_bounds__(kRowLaunch, 3)   // three 256-thread blocks per SM
k_scalogram(DevPlan P, const float2* __restrict__ xh, float* __restrict__ u1,
            float2* __restrict__ uh, float* __restrict__ s1) {
  extern __shared__ float2 sm[];
  const int lam = blockIdx.x, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  float* su = reinterpret_cast<float*>(sm + R.L + (R.L >> 4));   // after the padded row
  fold_first_order(P, R, xh + (size_t)b * (P.N >> 1), sm);
  __syncthreads();
  fft_dit_rows_r16<+1>(sm, R.logL, 1, twl_for(P, R.logL));
  const float invN = 1.f / (float)P.N;
  float* ub = u1 + (size_t)b * P.u1_len + R.off_u;
  for (int m = threadIdx.x; m < R.L; m += blockDim.x) {
    const float2 z = sm[fft_pos(m, R.logL)];
    const float a = hypotf(z.x, z.y) * invN;
    ub[m] = a;
    su[m] = a;
  }
  __syncthreads();
  // the row again, bit-reversed, for the forward FFT
  for (int m = threadIdx.x; m < R.L; m += blockDim.x)
    sm[fft_pos(bitrev(m, R.logL), R.logL)] = make_float2(su[m], 0.f);
  __syncthreads();
  fft_dit_rows_r16<-1>(sm, R.logL, 1, twl_for(P, R.logL));
  float2* hb = uh + (size_t)b * P.uh_len + R.off_uh;
  for (int k = threadIdx.x; k < (R.L >> 1); k += blockDim.x) hb[k] = sm[fft_pos(k, R.logL)];
  // S1[lambda, t] = sum_m s phi_T[(tT - m s) mod N] U1[m] from the row spectrum: with tau =
  // T / s, it is s (phi_s * U1)[t tau] for phi_s[j] = phi_T[j s], whose length-L DFT is
  // (1 / s) sum_r phi-hat[k + r L]; so S1[t] = (1 / L) sum_k Phi[k] U1-hat[k] e^{2 pi i k t / n_t}
  // with Phi[k] = sum_r phi-hat[k + r L], nonzero only near k = 0 (and L).  U1 is real: the
  // bins 0 < k < L / 2 count twice.  One warp per frame, lanes over the bins.
  {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int half = R.L >> 1;
    // bins [0, kA] near 0, and [kB, half] whose alias L - k is within phi-hat's support
    const int kA = min(half, P.phiT_kmax), kB = max(kA + 1, R.L - min(P.phiT_kmax, (P.N >> 1) - 1));
    const int nbins = kA + 1 + max(0, half - kB + 1);
    for (int t = w; t < P.n_t; t += nw) {
      float acc = 0.f;
      for (int i = l; i < nbins; i += 32) {
        const int k = i <= kA ? i : kB + (i - kA - 1);
        // signed representatives k + r L of the N-grid bins (the negative ones below Nyquist)
        float ph = 0.f;
        const int qneg = min(P.phiT_kmax, (P.N >> 1) - 1);
        for (int q = k; q <= P.phiT_kmax; q += R.L) ph += __ldg(&P.phiThat[q]);
        for (int q = R.L - k; q <= qneg; q += R.L) ph += __ldg(&P.phiThat[q]);
        if (ph == 0.f) continue;
        const float2 u = sm[fft_pos(k, R.logL)];
        float sn, cs;
        sincospif(2.f * (float)((k * t) & (P.n_t - 1)) / (float)P.n_t, &sn, &cs);
        acc += ((k == 0 || k == half) ? 1.f : 2.f) * ph * (u.x * cs - u.y * sn);
      }
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (l == 0) s1[((size_t)b * P.n1 + lam) * P.n_t + t] = acc / (float)R.L;
    }
  }
}

// ---------------------------------------------------------------------------------------
// Joint stage on CUDA cores (the plain FP32 comparison form).  One CTA per (c, alpha, b).
// Tile: all n1 rows x 32 time columns.  Thread (ty, tx) owns rows ty + 32 i, columns 4 tx + j.
// ---------------------------------------------------------------------------------------
constexpr int kJT = 256;      // threads
constexpr int kNC = 32;       // time columns per tile
constexpr int kRPT = 8;       // rows per thread (n1 <= 256)
constexpr int kPQ = 32;       // pooled (row, frame) accumulators per thread (n1 * n_t <= 8192)

struct JointSmem {
  float2* h;      // [N_fr]
  float2* yt;     // [n1][kNC]
  float* az;      // [n1][kNC + 1]
  float* wt;      // [n_t][kNC]
};

__global__ void __launch_bounds__(kJT)
k_joint_fwd_simt(DevPlan P, const float2* __restrict__ y, float* __restrict__ s2) {
  extern __shared__ float4 smraw[];
  const int c = blockIdx.x, a = blockIdx.y, b = blockIdx.z;
  const Rate2 A = P.rates2[a];
  float* out = s2 + (size_t)b * P.s2_stride + ((size_t)a * P.C + c) * P.n_lo * P.n_t;
  if (A.s == 0) {
    for (int i = threadIdx.x; i < P.n_lo * P.n_t; i += blockDim.x) out[i] = 0.f;
    return;
  }
  const int n1 = P.n1, nt = P.n_t, K = A.K, l0 = A.lam_min;
  float2* sh = reinterpret_cast<float2*>(smraw);
  float2* yt = sh + P.N_fr;
  float* az = reinterpret_cast<float*>(yt + (size_t)n1 * kNC);
  float* wt = az + (size_t)n1 * (nt > kNC + 1 ? nt : kNC + 1);
  for (int i = threadIdx.x; i < P.N_fr; i += blockDim.x) sh[i] = P.h[(size_t)c * P.N_fr + i];
  const int ty = threadIdx.x >> 3, tx = threadIdx.x & 7;
  const int nfm = P.N_fr - 1;
  float pacc[kPQ];
#pragma unroll
  for (int q = 0; q < kPQ; ++q) pacc[q] = 0.f;
  const float2* ya = y + (size_t)b * P.y_len + A.off_y;
  for (int n0 = 0; n0 < A.L; n0 += kNC) {
    __syncthreads();
    for (int i = threadIdx.x; i < K * kNC; i += blockDim.x) {
      const int k = i / kNC, col = i % kNC;
      yt[i] = (n0 + col < A.L) ? ya[(size_t)k * A.L + n0 + col] : make_float2(0.f, 0.f);
    }
    for (int i = threadIdx.x; i < nt * kNC; i += blockDim.x) {
      const int t = i / kNC, col = i % kNC;
      const int n = n0 + col;
      wt[i] = (n < A.L) ? __ldg(&P.phiT[(t * P.T - n * A.s) & (P.N - 1)]) * (float)A.s : 0.f;
    }
    __syncthreads();
    float2 acc[kRPT][4];
#pragma unroll
    for (int i = 0; i < kRPT; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
      const float4 y01 = reinterpret_cast<const float4*>(yt + k * kNC)[tx * 2];
      const float4 y23 = reinterpret_cast<const float4*>(yt + k * kNC)[tx * 2 + 1];
      const float2 yv[4] = {make_float2(y01.x, y01.y), make_float2(y01.z, y01.w),
                            make_float2(y23.x, y23.y), make_float2(y23.z, y23.w)};
      const int kk = k + l0;
#pragma unroll
      for (int i = 0; i < kRPT; ++i) {
        const int r = ty + 32 * i;
        if (r < n1) {
          const float2 hv = sh[(r - kk) & nfm];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x += hv.x * yv[j].x - hv.y * yv[j].y;
            acc[i][j].y += hv.x * yv[j].y + hv.y * yv[j].x;
          }
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kRPT; ++i) {
      const int r = ty + 32 * i;
      if (r < n1)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          az[r * (kNC + 1) + tx * 4 + j] = sqrtf(acc[i][j].x * acc[i][j].x + acc[i][j].y * acc[i][j].y);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kPQ; ++q) {
      const int p = threadIdx.x + q * kJT;
      if (p < n1 * nt) {
        const int r = p / nt, t = p % nt;
        const float* zr = az + r * (kNC + 1);
        const float* wr = wt + t * kNC;
        float s = 0.f;
#pragma unroll 8
        for (int col = 0; col < kNC; ++col) s += zr[col] * wr[col];
        pacc[q] += s;
      }
    }
  }
  __syncthreads();
  // time-pooled rows -> shared, then phi_F pooling along lambda (or none for Eq. 4)
  float* pm = az;  // [n1][n_t]
#pragma unroll
  for (int q = 0; q < kPQ; ++q) {
    const int p = threadIdx.x + q * kJT;
    if (p < n1 * nt) pm[p] = pacc[q];
  }
  __syncthreads();
  if (P.average_fr) {
    for (int i = threadIdx.x; i < P.n_lo * nt; i += blockDim.x) {
      const int lo = i / nt, t = i % nt;
      float s = 0.f;
      for (int r = 0; r < n1; ++r) s += __ldg(&P.phiF[(lo * P.s_F - r) & nfm]) * pm[r * nt + t];
      out[i] = s;
    }
  } else {
    for (int i = threadIdx.x; i < n1 * nt; i += blockDim.x) out[i] = pm[i];
  }
}

// Transposed FP32 Y planes for the TF32 contraction (its MMAs take K-major operands only):
// yt[alpha][2 b + part][n][lambda' - (lam_min & ~7)] = y[alpha][2 b + part][lambda' - lam_min][n],
// rounded to TF32, zero for lam_min & ~7 <= lambda' < lam_min and in the padding up to kt.  32 x 32 tiles
// through shared memory; grid (ceil(L / 32), ceil(kt / 32), 2 B) for one rate.
__global__ void k_transpose_yt(DevPlan P, int a, const float* __restrict__ y,
                               float* __restrict__ yt, int B) {
  __shared__ float tile[32][33];
  const Rate2 A = P.rates2[a];
  const int lm8 = A.lam_min & ~7;
  const int n0 = blockIdx.x * 32, c0 = blockIdx.y * 32, bp = blockIdx.z;
  const size_t plane = (size_t)A.K * A.L, tplane = (size_t)A.L * A.kt;
  const float* src = y + (size_t)B * 2 * A.off_y + (size_t)bp * plane;
  float* dst = yt + (size_t)B * 2 * A.off_yt + (size_t)bp * tplane;
  const int tx = threadIdx.x;
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int lp = lm8 + c0 + ty, n = n0 + tx;          // lambda' row, sample column
    float v = 0.f;
    if (lp >= A.lam_min && lp < P.n1 && n < A.L) v = src[(size_t)(lp - A.lam_min) * A.L + n];
    tile[ty][tx] = v;
  }
  __syncthreads();
  for (int ty = threadIdx.y; ty < 32; ty += blockDim.y) {
    const int n = n0 + ty, c = c0 + tx;
    if (n < A.L && c < A.kt) dst[(size_t)n * A.kt + c] = umma::tf32_rna(tile[tx][ty]);
  }
}

// Time scattering (Scattering1D, the baseline of Sec. 4.4): the second order without the
// log-frequency stage, S2t[alpha][lambda'][t] = sum_m s_alpha phi_T[(t T - m s_alpha) mod N]
// |Y_alpha[lambda'][m]|.  One CTA per G rows of one rate: the rows are folded and inverse
// transformed in shared memory as for the Y producer, their moduli replace them there, and
// each warp reduces one (row, frame) output at a time; Y never leaves the chip.
__global__ void __launch_bounds__(kRowBound)
k_scat1d_rows(DevPlan P, const int4* __restrict__ items, const float2* __restrict__ uh,
              float* __restrict__ s2t) {
  extern __shared__ float2 sm[];
  __shared__ int s_off[kMaxRowsPerItem], s_kend[kMaxRowsPerItem];
  __shared__ float s_inv[kMaxRowsPerItem];
  const int4 it = items[blockIdx.x];
  const int a = it.x, lam0 = it.y, G = it.z, b = blockIdx.y;
  const Rate2 A = P.rates2[a];
  const int L = A.L, logL = A.logL, nt = P.n_t;
  second_order_rows_ifft(P, A, a, lam0, G, uh + (size_t)b * P.uh_len, sm, s_off, s_kend, s_inv);
  __syncthreads();
  for (int idx = threadIdx.x; idx < G * L; idx += blockDim.x) {
    const float2 v = sm[fft_pos(idx, logL)];
    sm[fft_pos(idx, logL)].x = sqrtf(v.x * v.x + v.y * v.y) * s_inv[idx >> logL];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int o = warp; o < G * nt; o += nw) {
    const int r = o / nt, t = o - r * nt;
    float acc = 0.f;
    for (int m = lane; m < L; m += 32)
      acc = fmaf(__ldg(&P.phiT[((long long)t * P.T - (long long)m * A.s) & (P.N - 1)]),
                 sm[fft_pos((r << logL) + m, logL)].x, acc);
    for (int q = 16; q > 0; q >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, q);
    if (lane == 0)
      s2t[(((size_t)b * P.n2 + a) * P.n1 + lam0 + r) * nt + t] = acc * (float)A.s;
  }
}

// cudaFuncSetAttribute acts on the current device only, so the raised shared-memory limits
// are recorded per device (the plan's device is current in every call that launches).
std::mutex g_attrs_mu;
bool g_attrs_set[256] = {};

jtfs_status set_attrs(const jtfs_plan* p) {
  if (p->device < 0 || p->device >= 256) {
    set_error("device ordinal out of range");
    return JTFS_ERR_INVALID_ARG;
  }
  std::lock_guard<std::mutex> lk(g_attrs_mu);
  if (g_attrs_set[p->device]) return JTFS_OK;
  const int big = 227 * 1024;
  jtfs_status st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_xfft_sub, cudaFuncAttributeMaxDynamicSharedMemorySize, big), "attr")) != JTFS_OK) return st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_scalogram, cudaFuncAttributeMaxDynamicSharedMemorySize, big), "attr")) != JTFS_OK) return st;
  // the row producer holds at most 2^14 complex samples (padded one per 16) next to its
  // static row tables
  const int rows_smem = 140 * 1024;
  if ((st = cuda_check(cudaFuncSetAttribute(k_second_order_rows<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem), "attr")) != JTFS_OK) return st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_second_order_rows<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem), "attr")) != JTFS_OK) return st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_second_order_rows<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem), "attr")) != JTFS_OK) return st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_joint_fwd_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, big), "attr")) != JTFS_OK) return st;
  if ((st = cuda_check(cudaFuncSetAttribute(k_scat1d_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, rows_smem), "attr")) != JTFS_OK) return st;
  g_attrs_set[p->device] = true;
  return JTFS_OK;
}

}  // namespace

size_t joint_fwd_smem(const jtfs_plan* p) {
  const size_t azw = (size_t)(p->n_t > kNC + 1 ? p->n_t : kNC + 1);
  return (size_t)p->N_fr * 8 + (size_t)p->n1 * kNC * 8 + (size_t)p->n1 * azw * 4 +
         (size_t)p->n_t * kNC * 4;
}

bool joint_simt_supported(const jtfs_plan* p) {
  return p->n1 <= 32 * kRPT && (long long)p->n1 * p->n_t <= (long long)kPQ * kJT &&
         joint_fwd_smem(p) <= 227 * 1024;
}

// Autotuner of the Y producer (the largest FFT stage): times every (threads per CTA, samples
// per CTA) candidate on the plan's own work items for a batch of B signals, three launches
// each after one warm-up, with CUDA events on the stream, and keeps the fastest.  Candidates:
// 256 or 512 threads; 4096, 8192 or 16384 samples (at least the longest row).
jtfs_status autotune_rows(jtfs_plan* p, int B, const Workspace& w, cudaStream_t st,
                          int* best_threads, int* best_cap, float* best_ms) {
  jtfs_status rc = set_attrs(p);
  if (rc != JTFS_OK) return rc;
  const DevPlan& d = p->dp;
  std::vector<int> caps;
  for (int c : {4096, 8192, 16384}) {
    const int cap = std::max(c, p->L2max);
    if (cap <= 16384 && std::find(caps.begin(), caps.end(), cap) == caps.end()) caps.push_back(cap);
  }
  size_t most = 4;
  std::vector<std::vector<int>> tables;
  for (int cap : caps) {
    tables.push_back(build_rowitems(p, cap));
    most = std::max(most, tables.back().size());
  }
  int* d_items = nullptr;
  if ((rc = cuda_check(cudaMalloc(&d_items, most * sizeof(int)), "autotune items")) != JTFS_OK) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  int bt = p->row_threads, bc = p->rows_cap;
  for (size_t ci = 0; ci < caps.size() && rc == JTFS_OK; ++ci) {
    const std::vector<int>& items = tables[ci];
    if (items.empty()) continue;
    rc = cuda_check(cudaMemcpyAsync(d_items, items.data(), items.size() * sizeof(int),
                                    cudaMemcpyHostToDevice, st), "autotune upload");
    for (int threads : {256, 512}) {
      if (rc != JTFS_OK) break;
      auto launch = [&]() {
        const dim3 grid((unsigned)(items.size() / 4), B);
        const size_t smem = (size_t)caps[ci] * 17 / 2;   // padded one per 16
        if (p->use_tc)
          k_second_order_rows<1><<<grid, threads, smem, st>>>(
              d, reinterpret_cast<const int4*>(d_items), w.uh, nullptr, (__nv_bfloat16*)w.ybh,
              (__nv_bfloat16*)w.ybl, B);
        else
          k_second_order_rows<0><<<grid, threads, smem, st>>>(
              d, reinterpret_cast<const int4*>(d_items), w.uh, w.y, nullptr, nullptr, B);
      };
      launch();
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3; ++r) launch();
      cudaEventRecord(e1, st);
      if ((rc = cuda_check(cudaEventSynchronize(e1), "autotune timing")) != JTFS_OK) break;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) { best = ms; bt = threads; bc = caps[ci]; }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_items);
  if (rc != JTFS_OK) return rc;
  // install the winner's item table
  std::vector<int> items = build_rowitems(p, bc);
  if (p->d_rowitems_own) { cudaFree(p->d_rowitems_own); p->d_rowitems_own = nullptr; }
  if ((rc = cuda_check(cudaMalloc(&p->d_rowitems_own, std::max<size_t>(16, items.size() * sizeof(int))), "tuned items")) != JTFS_OK)
    return rc;
  if ((rc = cuda_check(cudaMemcpy(p->d_rowitems_own, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice), "tuned items")) != JTFS_OK)
    return rc;
  p->rowitems = items;
  p->d_rowitems = (int*)p->d_rowitems_own;
  p->rows_cap = bc;
  p->row_threads = bt;
  *best_threads = bt;
  *best_cap = bc;
  *best_ms = best / 3.f;
  return JTFS_OK;
}


// Time scattering forward: the first order as in the transform (S0, S1, the U1 checkpoint and
// its row spectra), then the second-order moduli pooled per (alpha, lambda') path.  s2t is
// [B][n2][n1][n_t], zero outside the paths (skipped rates, rows below lam_min).
jtfs_status launch_scat1d_forward(const jtfs_plan* p, const float* x, int B, float* s0, float* s1,
                                  float* s2t, float* u1, const Workspace& w, cudaStream_t st) {
  jtfs_status rc = set_attrs(p);
  if (rc != JTFS_OK) return rc;
  const DevPlan& d = p->dp;
  {
    StageScope sc(p, kStXfft, st, 2);
    k_xfft_sub<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, x, w.xsub);
    k_xfft_combine<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.xsub, w.xh);
  }
  {
    StageScope sc(p, kStS0, st, 1);
    k_s0<<<dim3(kS0Split * p->n_t, B), kS0Threads, 0, st>>>(d, x, s0);
  }
  {
    StageScope sc(p, kStScalogram, st, 1);
    k_scalogram<<<dim3(p->n1, B), kRowLaunch, (size_t)p->L1max * 17 / 2 + (size_t)p->L1max * 4, st>>>(d, w.xh, u1, w.uh, s1);
  }
  if ((rc = cuda_check(cudaMemsetAsync(s2t, 0, (size_t)B * p->n2 * p->n1 * p->n_t * sizeof(float), st), "memset")) != JTFS_OK)
    return rc;
  if (!p->rowitems.empty()) {
    StageScope sc(p, kStSecondOrder, st, 1);
    k_scat1d_rows<<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                    (size_t)p->rows_cap * 17 / 2, st>>>(
        d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, s2t);
  }
  return cuda_check(cudaGetLastError(), "time scattering forward");
}

jtfs_status launch_forward(const jtfs_plan* p, const float* x, int B, float* s0, float* s1,
                           float* s2, float* u1, const Workspace& w, cudaStream_t st) {
  jtfs_status rc = set_attrs(p);
  if (rc != JTFS_OK) return rc;
  const DevPlan& d = p->dp;
  {
    StageScope sc(p, kStXfft, st, 2);
    k_xfft_sub<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, x, w.xsub);
    k_xfft_combine<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, w.xsub, w.xh);
  }
  {
    StageScope sc(p, kStS0, st, 1);
    k_s0<<<dim3(kS0Split * p->n_t, B), kS0Threads, 0, st>>>(d, x, s0);
  }
  {
    StageScope sc(p, kStScalogram, st, 1);
    k_scalogram<<<dim3(p->n1, B), kRowLaunch, (size_t)p->L1max * 17 / 2 + (size_t)p->L1max * 4, st>>>(d, w.xh, u1, w.uh, s1);
  }
  if (p->use_tc && p->cfg.precision == JTFS_PREC_TF32) {
    // TF32 operands: Y as FP32 planes (in the complex FP32 buffer, same size)
    if (!p->pairs.empty()) {
      StageScope sc(p, kStSecondOrder, st, 1);
      k_second_order_rows<2><<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                              (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, w.y, nullptr, nullptr, B);
    }
    {
      StageScope sc(p, kStSecondOrder, st, 0);
      for (int a = 0; a < p->n2; ++a) {
        const Rate2& A = p->rates2[a];
        if (A.s == 0 || A.kt == 0) continue;
        k_transpose_yt<<<dim3((A.L + 31) / 32, (A.kt + 31) / 32, 2 * B), dim3(32, 8), 0, st>>>(
            d, a, reinterpret_cast<const float*>(w.y), w.yt, B);
        ++p->prof.launches;
      }
    }
    StageScope sc(p, kStJointFwd, st, 0);   // the launcher counts its kernels
    jtfs_status r2 = launch_joint_fwd_tc(p, B, w.yt, nullptr, w.pbuf, s2, st);
    if (r2 != JTFS_OK) return r2;
  } else if (p->use_tc) {
    if (!p->pairs.empty()) {
      StageScope sc(p, kStSecondOrder, st, 1);
      k_second_order_rows<1><<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                              (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, nullptr,
          (__nv_bfloat16*)w.ybh, (__nv_bfloat16*)w.ybl, B);
    }
    StageScope sc(p, kStJointFwd, st, 0);   // the launcher counts its kernels
    jtfs_status r2 = launch_joint_fwd_tc(p, B, w.ybh, w.ybl, w.pbuf, s2, st);
    if (r2 != JTFS_OK) return r2;
  } else {
    if (!p->pairs.empty()) {
      StageScope sc(p, kStSecondOrder, st, 1);
      k_second_order_rows<0><<<dim3((unsigned)(p->rowitems.size() / 4), B), p->row_threads,
                              (size_t)p->rows_cap * 17 / 2, st>>>(
          d, reinterpret_cast<const int4*>(p->d_rowitems), w.uh, w.y, nullptr, nullptr, B);
    }
    StageScope sc(p, kStJointFwd, st, 1);
    k_joint_fwd_simt<<<dim3(p->C, p->n2, B), kJT, joint_fwd_smem(p), st>>>(d, w.y, s2);
  }
  return cuda_check(cudaGetLastError(), "forward launch");
}

}  // namespace jtfs

// ---------------------------------------------------------------------------------------
// First-order transform (S0, S1) without any device allocation.
//
// Some callers cannot allocate device memory while they run: a real-time audio callback,
// where cudaMalloc may block for milliseconds and miss the audio deadline, or a plug-in
// hosted inside an application that owns and budgets all of the device's memory.  For
// them the scratch of this path (the decimated spectra, x-hat, the scalogram rows and their
// spectra) lives in one fixed array compiled into the library.  That array is held by every
// GPU that loads the library until the process exits, and every call shares it: calls that
// overlap on the GPU (other streams, other host threads) race on it.  Each kernel here
// writes every scratch element it later reads, so nothing has to be cleared between calls.
// ---------------------------------------------------------------------------------------

namespace jtfs {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB per device
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
void* g_static_ptr[256] = {};
}  // namespace

size_t first_order_static_bytes(const jtfs_plan* p, int64_t B) {
  auto a = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t Bz = (size_t)B;
  return a(Bz * p->N * 8) + a(Bz * (p->N / 2) * 8) + a(Bz * p->u1_len * 4) + a(Bz * p->uh_len * 8);
}

// The array's device address, looked up once per device with that device current (the
// name of the array is only a host-side stand-in in host code).
jtfs_status static_scratch(int dev, void** out) {
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (dev < 0 || dev >= 256) {
    set_error("device ordinal out of range");
    return JTFS_ERR_INVALID_ARG;
  }
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    jtfs_status st = cuda_check(cudaGetSymbolAddress(&ptr, g_static_scratch), "cudaGetSymbolAddress");
    if (st != JTFS_OK) return st;
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return JTFS_OK;
}

jtfs_status launch_first_order_static(const jtfs_plan* p, const float* x, int B, float* s0,
                                      float* s1, cudaStream_t st) {
  const size_t need = first_order_static_bytes(p, B);
  if (need > kStaticScratchBytes) {
    set_error("jtfs_first_order_static: B = " + std::to_string(B) + " needs " +
              std::to_string(need) + " bytes of scratch; the fixed array holds " +
              std::to_string(kStaticScratchBytes) + " (use a smaller batch or jtfs_forward)");
    return JTFS_ERR_WORKSPACE;
  }
  void* base = nullptr;
  jtfs_status rc = static_scratch(p->device, &base);
  if (rc != JTFS_OK) return rc;
  if ((rc = set_attrs(p)) != JTFS_OK) return rc;
  auto a = [](size_t v) { return (v + 255) & ~(size_t)255; };
  const size_t Bz = (size_t)B;
  char* c = (char*)base;
  float2* xsub = (float2*)c;
  c += a(Bz * p->N * 8);
  float2* xh = (float2*)c;
  c += a(Bz * (p->N / 2) * 8);
  float* u1 = (float*)c;
  c += a(Bz * p->u1_len * 4);
  float2* uh = (float2*)c;
  const DevPlan& d = p->dp;
  k_xfft_sub<<<dim3(d.D, B), kFftThreads, (size_t)d.M * 17 / 2, st>>>(d, x, xsub);
  k_xfft_combine<<<dim3((p->N / 2 + 255) / 256, B), 256, 0, st>>>(d, xsub, xh);
  k_s0<<<dim3(kS0Split * p->n_t, B), kS0Threads, 0, st>>>(d, x, s0);
  k_scalogram<<<dim3(p->n1, B), kRowLaunch, (size_t)p->L1max * 17 / 2 + (size_t)p->L1max * 4, st>>>(d, xh, u1, uh, s1);
  return cuda_check(cudaGetLastError(), "first-order static launch");
}

}  // namespace jtfs

extern "C" jtfs_status jtfs_first_order_static(const jtfs_plan* p, const float* x, int64_t B,
                                               float* s0, float* s1, void* stream) {
  using namespace jtfs;
  if (!p || B < 0 || B > (1 << 20)) {
    set_error("bad plan or batch size");
    return JTFS_ERR_INVALID_ARG;
  }
  if (B == 0) return JTFS_OK;
  if (!x || !s0 || !s1) {
    set_error("NULL input or output");
    return JTFS_ERR_INVALID_ARG;
  }
  int dev = -1;
  jtfs_status st = cuda_check(cudaGetDevice(&dev), "cudaGetDevice");
  if (st != JTFS_OK) return st;
  if (dev != p->device) {
    set_error("current device differs from the plan's device");
    return JTFS_ERR_INVALID_ARG;
  }
  return launch_first_order_static(p, x, (int)B, s0, s1, (cudaStream_t)stream);
}
