// The phi_t paths of the second order and the 2-D output layout, on CUDA cores, FP32.
//
// Eq. 3 with the time lowpass phi_T in place of the time wavelet psi_alpha: the joint filters
// phi_T(t) psi_{beta,+1}(lambda) (PHI_PSI) and phi_T(t) phi_F(lambda) (PHI_PHI).  Their time
// filter's band [0, 4 sigma_T] is sampled like a time wavelet's band, at stride T for
// oversampling 0, and the first-order rows filtered by phi_T and sampled every T samples are
// exactly S1 (the Riemann sums of phi_T at each row's stride).  So a path is
//   Z = W_c S1 (zero-padded convolution along lambda; W_c real for phi_F),
//   S = P_F |Z| P_T^T, with P_T the Riemann sum of phi_T at stride T (a circulant over the
//   n_t frames) and P_F the phi_F pooling (identity for Eq. 4),
// and its adjoint is a cotangent of S1: Re(W_c^H (g_|Z| Z / |Z|)) with g_|Z| = P_F^T g P_T.
// The input S1 being real, the spin-down filter gives Z's conjugate and the same modulus, so
// one spin is kept.
//
//   k_phi_fwd      : per (path, signal): the path from S1 into the tail of the signal's S2
//   k_phi_bwd      : per signal: g_S1 + the adjoint of every path
//   k_s1_from_u1   : per (lambda, signal): S1 from the U1 checkpoint (Riemann sums in time),
//                    for a backward call that did not run the forward
//   k_pack_2d      : the 2-D layout, [out_rows][n_t] per signal: S0, S1 rows, S2 paths
#include <algorithm>

#include "internal.h"

namespace jtfs {
namespace {

constexpr int kPhiThreads = 256;

__device__ __forceinline__ int path_channel(const DevPlan& P, int q) {
  return (P.phi_psi && q < P.n_fr) ? q : 2 * P.n_fr;
}

// Z = W_c Y at (lam, m) for a block-resident Y [n1][nt] and h_c [N_fr].
__device__ __forceinline__ float2 lambda_conv(const float2* h, const float* y, int n1, int nt,
                                              int nfm, int lam, int m) {
  float zr = 0.f, zi = 0.f;
  for (int lp = 0; lp < n1; ++lp) {
    const float2 hv = h[(lam - lp) & nfm];
    const float v = y[lp * nt + m];
    zr = fmaf(hv.x, v, zr);
    zi = fmaf(hv.y, v, zi);
  }
  return make_float2(zr, zi);
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi_fwd(DevPlan P, const float* __restrict__ s1, float* __restrict__ s2) {
  extern __shared__ float2 sm2[];
  const int q = blockIdx.x, b = blockIdx.y;
  const int n1 = P.n1, nt = P.n_t, nfm = P.N_fr - 1, cells = n1 * nt;
  const int c = path_channel(P, q);
  float2* h = sm2;                                    // [N_fr]
  float* y = reinterpret_cast<float*>(h + P.N_fr);    // [n1][nt] S1, then the time-pooled rows
  float* az = y + cells;                              // [n1][nt] |Z|
  float* wt = az + cells;                             // [nt] T phi_T[d T]
  const float* src = s1 + (size_t)b * cells;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) y[i] = src[i];
  for (int i = threadIdx.x; i < nt; i += blockDim.x)
    wt[i] = (float)P.T * __ldg(&P.phiT[((long long)i * P.T) & (P.N - 1)]);
  for (int i = threadIdx.x; i < P.N_fr; i += blockDim.x) h[i] = P.h[(size_t)c * P.N_fr + i];
  __syncthreads();
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    const int lam = i / nt, m = i - lam * nt;
    const float2 z = lambda_conv(h, y, n1, nt, nfm, lam, m);
    az[i] = sqrtf(z.x * z.x + z.y * z.y);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    const int lam = i / nt, t = i - lam * nt;
    float acc = 0.f;
    for (int m = 0; m < nt; ++m) acc = fmaf(wt[(t - m) & (nt - 1)], az[lam * nt + m], acc);
    y[i] = acc;
  }
  __syncthreads();
  float* out = s2 + (size_t)b * P.s2_stride + ((size_t)P.n2 * P.C + q) * P.n_lo * nt;
  for (int i = threadIdx.x; i < P.n_lo * nt; i += blockDim.x) {
    if (!P.average_fr) {
      out[i] = y[i];
      continue;
    }
    const int lo = i / nt, t = i - lo * nt;
    float acc = 0.f;
    for (int r = 0; r < n1; ++r)
      acc = fmaf(__ldg(&P.phiF[(lo * P.s_F - r) & nfm]), y[r * nt + t], acc);
    out[i] = acc;
  }
}

__global__ void __launch_bounds__(kPhiThreads)
k_phi_bwd(DevPlan P, const float* __restrict__ s1, const float* __restrict__ gs2,
          const float* __restrict__ gs1, float* __restrict__ gs1_out) {
  extern __shared__ float2 sm2[];
  const int b = blockIdx.x;
  const int n1 = P.n1, nt = P.n_t, nfm = P.N_fr - 1, cells = n1 * nt;
  float2* h = sm2;                                    // [N_fr]
  float* y = reinterpret_cast<float*>(h + P.N_fr);    // [n1][nt] S1
  float* gy = y + cells;                              // [n1][nt] cotangent of S1
  float* gr = gy + cells;                             // [n1][nt] g_|Z|, then Re gZ
  float* gi = gr + cells;                             // [n1][nt] lambda-pooling adjoint, then Im gZ
  float* wt = gi + cells;                             // [nt]
  const float* src = s1 + (size_t)b * cells;
  for (int i = threadIdx.x; i < cells; i += blockDim.x) {
    y[i] = src[i];
    gy[i] = gs1 ? gs1[(size_t)b * cells + i] : 0.f;
  }
  for (int i = threadIdx.x; i < nt; i += blockDim.x)
    wt[i] = (float)P.T * __ldg(&P.phiT[((long long)i * P.T) & (P.N - 1)]);
  for (int q = 0; q < P.n_phi; ++q) {
    const int c = path_channel(P, q);
    const float* g = gs2 + (size_t)b * P.s2_stride + ((size_t)P.n2 * P.C + q) * P.n_lo * nt;
    __syncthreads();   // the previous path is done with h, gr, gi
    for (int i = threadIdx.x; i < P.N_fr; i += blockDim.x) h[i] = P.h[(size_t)c * P.N_fr + i];
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lam = i / nt, t = i - lam * nt;
      float acc = 0.f;
      if (P.average_fr) {
        for (int lo = 0; lo < P.n_lo; ++lo)
          acc = fmaf(__ldg(&P.phiF[(lo * P.s_F - lam) & nfm]), g[lo * nt + t], acc);
      } else {
        acc = g[i];
      }
      gi[i] = acc;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lam = i / nt, m = i - lam * nt;
      float acc = 0.f;
      for (int t = 0; t < nt; ++t) acc = fmaf(wt[(t - m) & (nt - 1)], gi[lam * nt + t], acc);
      gr[i] = acc;
    }
    __syncthreads();
    // gZ = g_|Z| Z / |Z| (0 where Z = 0), each cell in place
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lam = i / nt, m = i - lam * nt;
      const float2 z = lambda_conv(h, y, n1, nt, nfm, lam, m);
      const float a = sqrtf(z.x * z.x + z.y * z.y);
      const float s = a > 0.f ? gr[i] / a : 0.f;
      gr[i] = s * z.x;
      gi[i] = s * z.y;
    }
    __syncthreads();
    // g_S1[lam'][m] += sum_lam Re(conj(h[lam - lam']) gZ[lam][m])
    for (int i = threadIdx.x; i < cells; i += blockDim.x) {
      const int lp = i / nt, m = i - lp * nt;
      float acc = 0.f;
      for (int lam = 0; lam < n1; ++lam) {
        const float2 hv = h[(lam - lp) & nfm];
        acc = fmaf(hv.x, gr[lam * nt + m], acc);
        acc = fmaf(hv.y, gi[lam * nt + m], acc);
      }
      gy[i] += acc;
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < cells; i += blockDim.x) gs1_out[(size_t)b * cells + i] = gy[i];
}

// S1[lam][t] = sum_m s phi_T[(t T - m s) mod N] U1_lam[m] for the row of stride s.
__global__ void k_s1_from_u1(DevPlan P, const float* __restrict__ u1, float* __restrict__ s1) {
  __shared__ float red[kPhiThreads / 32];
  const int lam = blockIdx.x, b = blockIdx.y;
  const Row1 R = P.rows1[lam];
  const float* row = u1 + (size_t)b * P.u1_len + R.off_u;
  for (int t = 0; t < P.n_t; ++t) {
    float acc = 0.f;
    for (int m = threadIdx.x; m < R.L; m += blockDim.x)
      acc = fmaf(__ldg(&P.phiT[((long long)t * P.T - (long long)m * R.s) & (P.N - 1)]), row[m], acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      float s = 0.f;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
      s1[((size_t)b * P.n1 + lam) * P.n_t + t] = s * (float)R.s;
    }
    __syncthreads();
  }
}

// The 2-D layout: per signal, row 0 = S0, rows 1..n1 = S1, then the S2 paths' n_lo rows each.
// unpack = 1 reads the packed buffer into the three separate ones (cotangents).
__global__ void k_pack_2d(DevPlan P, float* s0, float* s1, float* s2, float* out, int unpack) {
  const int b = blockIdx.y;
  const size_t n0 = P.n_t, n1 = (size_t)P.n1 * P.n_t, n2 = (size_t)P.s2_stride;
  const size_t per = n0 + n1 + n2;
  float* o = out + (size_t)b * per;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < per;
       i += (size_t)gridDim.x * blockDim.x) {
    float* sep = i < n0 ? s0 + (size_t)b * n0 + i
                        : (i < n0 + n1 ? s1 + (size_t)b * n1 + (i - n0)
                                       : s2 + (size_t)b * n2 + (i - n0 - n1));
    if (unpack) *sep = o[i]; else o[i] = *sep;
  }
}

size_t phi_fwd_smem(const jtfs_plan* p) {
  return (size_t)p->N_fr * 8 + (size_t)(2 * p->n1 * p->n_t + p->n_t) * 4;
}
size_t phi_bwd_smem(const jtfs_plan* p) {
  return (size_t)p->N_fr * 8 + (size_t)(4 * p->n1 * p->n_t + p->n_t) * 4;
}

}  // namespace

bool phi_supported(const jtfs_plan* p) {
  // the phi_t paths' input is S1 itself only when phi_T's band is sampled at stride T
  // (oversampling 0); one block holds the paths' whole [n1][n_t] planes
  return p->cfg.oversampling == 0 && phi_bwd_smem(p) <= 227 * 1024;
}

jtfs_status launch_phi_forward(const jtfs_plan* p, int B, const float* s1, float* s2,
                               cudaStream_t st) {
  const size_t smem = phi_fwd_smem(p);
  jtfs_status rc = cuda_check(cudaFuncSetAttribute(k_phi_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
  if (rc != JTFS_OK) return rc;
  StageScope sc(p, kStJointFwd, st, 1);
  k_phi_fwd<<<dim3(p->n_phi, B), kPhiThreads, smem, st>>>(p->dp, s1, s2);
  return cuda_check(cudaGetLastError(), "k_phi_fwd");
}

jtfs_status launch_s1_from_u1(const jtfs_plan* p, int B, const float* u1, float* s1,
                              cudaStream_t st) {
  StageScope sc(p, kStUhFromU1, st, 1);
  k_s1_from_u1<<<dim3(p->n1, B), kPhiThreads, 0, st>>>(p->dp, u1, s1);
  return cuda_check(cudaGetLastError(), "k_s1_from_u1");
}

jtfs_status launch_phi_backward(const jtfs_plan* p, int B, const float* s1, const float* gs2,
                                const float* gs1, float* gs1_out, cudaStream_t st) {
  const size_t smem = phi_bwd_smem(p);
  jtfs_status rc = cuda_check(cudaFuncSetAttribute(k_phi_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem), "attr");
  if (rc != JTFS_OK) return rc;
  StageScope sc(p, kStJointBwd, st, 1);
  k_phi_bwd<<<B, kPhiThreads, smem, st>>>(p->dp, s1, gs2, gs1, gs1_out);
  return cuda_check(cudaGetLastError(), "k_phi_bwd");
}

jtfs_status launch_pack_2d(const jtfs_plan* p, int B, const float* s0, const float* s1,
                           const float* s2, float* out, bool unpack, cudaStream_t st) {
  const size_t per = (size_t)p->n_t * (1 + p->n1) + (size_t)p->dp.s2_stride;
  const int gx = (int)std::min<size_t>(64, (per + 255) / 256);
  StageScope sc(p, unpack ? kStJointBwd : kStJointFwd, st, 1);
  k_pack_2d<<<dim3(gx, B), 256, 0, st>>>(p->dp, const_cast<float*>(s0), const_cast<float*>(s1),
                                          const_cast<float*>(s2), out, unpack ? 1 : 0);
  return cuda_check(cudaGetLastError(), "k_pack_2d");
}

}  // namespace jtfs
